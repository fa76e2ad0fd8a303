#!/usr/bin/env python3
"""Throughput of the SIR time step (Alg. 1) for single-spot tracking on GB300.

Workload (the paper-scale plain SIR): N = 38,000,000 particles, state 6 x
float32 SoA, 512 x 512 float32 Poisson frames with one Gaussian-PSF spot
(sigma_PSF ~ U[1.2, 2.0], SNR ~ U[2, 8], seeded), 11 x 11 patch, groups of
4096 particles, resampling every frame.  One step = one frame: propagate,
likelihood, normalise + estimate, resample.  value = particle-steps / s over
all ranks; frames are resident in HBM before the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SIR particle-steps/sec at N=38M vs plain FP32; % of roofline; grad steps/sec"
UNIT = "particle-steps/s"
N_FULL = 38_000_000
GROUP = 4096
W = H = 512
R = 5
# algorithmic HBM bytes per particle of the fused step kernel after a global
# resample: ancestor 4 + gathered parent x, y, vx, vy, I0 20 + written state 24
STEP_BYTES = 48
# measured DRAM bytes per particle of the same kernel (ncu dram__bytes_read.sum +
# dram__bytes_write.sum, the 5th launch at N = 16M, the step kernel's summary under
# profiles/), scaled to a launch by N; set to None whenever step_kernel changes
STEP_TRAFFIC_PER_PARTICLE = (347167744 + 338496768) / 16e6
# algorithmic FP32 flops per particle of the likelihood + propagation (an FMA
# counts 2), two counts:
#  * the expanded form the kernel evaluates, l = I0 (B - I0 C / 2) / sigma_xi^2
#    with B, C separable patch sums: bilinear form 2P^2, row combination 2P,
#    sums of squares 4P, final combination 6, propagation 10, P = 2r + 1;
#  * the per-pixel form: model FMA, residual, accumulating FMA = 5 flops per
#    pixel over P^2 pixels (605 at r = 5)
STEP_FLOPS = 2 * 11 * 11 + 2 * 11 + 4 * 11 + 6 + 10
STEP_FLOPS_PER_PIXEL_FORM = 5 * 11 * 11
# unit-count FP32 peak (152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz), used
# only when the FMA-chain measurement cannot run
FP32_PEAK_DERIVED_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
TIMED_RUNS = 5


# the scheme rows, in the order they run in one context: every row starts
# from balanced groups except the LGS rows, which unbalance them themselves
SCHEME_ROWS = [("rpa_gs", 0.0), ("rpa_sgs", 0.0), ("rpa2_gs", 0.0), ("rpa2_sgs", 0.0), ("rna", 0.1), ("rna", 0.5),
               ("arna", 0.5), ("systematic", 0.0), ("rpa_lgs", 0.0), ("rpa2_lgs", 0.0)]


def workload_desc(n, scheme, target_n=None):
    d = {
        "workload": f"spot512: {W}x{H} float32 Poisson frames, one Gaussian-PSF spot, N={n:,} particles, "
                    f"{2 * R + 1}x{2 * R + 1} patch, groups of {GROUP}, {scheme} resampling every frame",
        "N": n, "frame": f"{W}x{H}", "patch": 2 * R + 1, "group_size": GROUP, "scheme": scheme,
        "state": "6 x float32 SoA (x, y, vx, vy, I0, lw), double-buffered",
        "l2": "inputs larger than L2: 1.8 GB of particle state per frame (no flush needed)",
    }
    if target_n is not None and target_n != n:
        d["target_N"] = target_n
    return d


def make_workload(k_total, seed=0):
    import synth
    mv, p = synth.preset("spot512_k50", seed=seed, K=k_total)
    params = dict(width=W, height=H, patch_radius=R, psf_sigma=float(p["sigma"]),
                  amplitude=float(p["amplitude"]), background=10.0, sigma_xi=math.sqrt(10.0),
                  sigma_m=0.5, sigma_v=0.1, sigma_I=1.0, v0_max=1.0)
    return mv, params


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0, period_ms=100):
        self.rows = []
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-i", str(device_index), "-lms", str(period_ms)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.t.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle legs
def cpu_model():
    """The host CPU's model name (x86 'model name', else lscpu's 'Model name')."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_rate(params, frames, n, k, threads, seed=0):
    """The FP64 oracle as it stands on n particles x k frames, with `threads`
    OpenMP threads over particles (results do not depend on the count).
    Returns (particle-steps/s, seconds, threads used)."""
    import oracle as orc
    used = orc.set_threads(threads)
    m = orc.Model(**{**params, "seed": seed})
    t0 = time.perf_counter()
    rc, est, _ = orc.run(m, n, frames[:k], group_size=GROUP, scheme=orc.SYSTEMATIC)
    dt = time.perf_counter() - t0
    return n * k / dt, dt, used


def cpu_baseline(params, frames, cn, ck):
    """The oracle on the host cores: the spot512 workload (n particles x k
    frames) on all cores, and the 128 x 128 workload in full (N = 16384,
    20 frames, 9 x 9 patch) on one core and on all cores."""
    import synth
    allc = os.cpu_count() or 1
    rate, dt, used = oracle_rate(params, frames, cn, ck, allc)
    mv1 = synth.make_movie(W=128, H=128, K=20, sigma=1.5, amplitude=50.0, background=10.0, seed=0)
    p1 = dict(width=128, height=128, patch_radius=4, psf_sigma=1.5, amplitude=50.0, background=10.0,
              sigma_xi=math.sqrt(10.0), sigma_m=0.5, sigma_v=0.1, sigma_I=1.0, v0_max=1.0)
    r1, d1, _ = oracle_rate(p1, mv1.frames, 16384, 20, 1)
    rm, dm, um = oracle_rate(p1, mv1.frames, 16384, 20, allc)
    return {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"FP64 C oracle, OpenMP over particles on {used} threads, {cn:,} particles x {ck} frames of "
                      f"the same workload ({dt:.1f} s)",
            "cpu_model": cpu_model(), "nproc": allc,
            "spot128_full": {"workload": "128x128, 20 frames, N=16384, 9x9 patch, systematic",
                             "single_thread": r1, "single_thread_s": d1, "all_cores": rm, "all_cores_s": dm,
                             "threads": um}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as orc
    n = args.ref_n
    used = orc.set_threads(os.cpu_count() or 1)
    mv, params = make_workload(args.warmup + args.steps + 1)
    m = orc.Model(**{**params, "seed": 0})
    st = orc.init(m, n)
    anc = np.arange(n, dtype=np.int32)
    lw_prev = np.zeros(n)
    G = (n + GROUP - 1) // GROUP
    goff = orc.balanced_offsets(n, G)
    ring = np.arange(G, dtype=np.int32)
    scheme = {"systematic": orc.SYSTEMATIC, "rpa_gs": orc.RPA_GS, "rpa_sgs": orc.RPA_SGS, "rpa_lgs": orc.RPA_LGS,
              "rna": orc.RNA, "rpa2_gs": orc.RPA2_GS, "rpa2_sgs": orc.RPA2_SGS, "rpa2_lgs": orc.RPA2_LGS,
              "arna": orc.ARNA}[args.scheme]
    alpha = float(np.float32(args.alpha))
    times = []
    for k in range(1, args.warmup + args.steps + 1):
        t0 = time.perf_counter()
        nxt = orc.propagate(m, k, st, anc, lw_prev)
        nxt = orc.weight(m, mv.frames[k - 1], nxt)
        so = orc.summary(nxt, lw_prev)
        lwf = nxt[5].astype(np.float32)
        if scheme == orc.ARNA:
            rc, anc, lw_prev, goff, _, ring = orc.resample_arna(m, n, k, goff, lwf, so["log_evidence"] < 0.0, ring,
                                                                lw_sum=nxt[5], alpha=alpha)
        else:
            rc, anc, lw_prev, goff, _ = orc.resample(m, scheme, n, k, goff, lwf, nxt[5], alpha=alpha)
        st = nxt
        if k > args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n * args.steps / total
    sample = (f"{n:,} particles of the same workload per step (one frame each), FP64, OpenMP over particles on "
              f"{used} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_desc(n, args.scheme, target_n=N_FULL),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- ranks
def max_over_ranks(t_ms, dist, device):
    """Barrier, then the largest of every rank's time: the job ends with its
    slowest rank."""
    if dist is None:
        return t_ms
    import torch
    dist.barrier()
    t = torch.tensor([t_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(n_per_rank, steps, world, t_ms):
    """Whole-job particle-steps/s: every rank's particles over the slowest
    rank's time."""
    return n_per_rank * steps * world / (t_ms / 1e3)


# ---------------------------------------------------------------- ours
def timed_frames(pf, frames, k0, K, scheme, alpha, stream):
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(k0, k0 + K):
        pf.step(frames[k - 1], k)
        pf.resample(scheme, alpha)
    ev1.record(stream)
    ev1.synchronize()
    return ev0.elapsed_time(ev1)


def spread_ab(ppf, params, rank, n, stream, args):
    """Frame 1 (the prior draw, spread over the whole frame) on each
    likelihood path; the first four frames with systematic resampling; and an
    ARNA run through a movie whose spot vanishes for ten frames (direct path
    forced against the automatic choice)."""
    import torch
    import synth
    out = {"workload": f"spot512 at N={n:,}: frame 1 from the prior; frames 1-4 with systematic resampling; and "
                       "5 frames, the spot gone for 10, 5 more (ARNA, maximum alpha 0.5)"}
    mv, _ = make_workload(20, seed=0)
    blank = synth.make_movie(W=W, H=H, K=20, sigma=1.5, amplitude=0.0, background=10.0, seed=99)
    frames = torch.from_numpy(mv.frames).cuda()
    lost = mv.frames.copy()
    lost[5:15] = blank.frames[5:15]
    lost = torch.from_numpy(lost).cuda()
    model = ppf.Model(**params, seed=rank, filter_id=rank)
    first = {}
    for name, path in (("direct", ppf.PATH_DIRECT), ("binned", ppf.PATH_BINNED), ("auto", ppf.PATH_AUTO)):
        pf = ppf.ParticleFilter(model, n, group_size=GROUP, stream=stream)
        pf.set_likelihood_path(path)
        torch.cuda.synchronize()
        pf.profile_enable(True, capacity=4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pf.step(frames[0], 1)
        e1.record(stream)
        e1.synchronize()
        pr = pf.profile_read()
        first[name] = {"ms": e0.elapsed_time(e1), "step_ms": pr["step_ms"], "binned": pf.last_step_binned()}
        pf.close()
    out["frame1"] = first
    # the first frames with systematic resampling: the draw after the spread
    # frame concentrates the cloud, so the automatic choice goes direct at once
    sysrun = {}
    for name, path in (("direct", ppf.PATH_DIRECT), ("auto", ppf.PATH_AUTO)):
        pf = ppf.ParticleFilter(model, n, group_size=GROUP, stream=stream)
        pf.set_likelihood_path(path)
        ms, binned = [], []
        for k in range(1, 5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pf.step(frames[k - 1], k)
            e1.record(stream)
            pf.resample(ppf.SYSTEMATIC)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            binned.append(pf.last_step_binned())
        sysrun[name] = {"step_ms_per_frame": ms, "binned": binned}
        pf.close()
    out["first_frames_systematic"] = sysrun
    lostrun = {}
    for name, path in (("direct", ppf.PATH_DIRECT), ("auto", ppf.PATH_AUTO)):
        pf = ppf.ParticleFilter(model, n, group_size=GROUP, stream=stream)
        pf.set_likelihood_path(path)
        ms, binned = [], []
        for k in range(1, 21):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pf.step(lost[k - 1], k)
            e1.record(stream)
            pf.resample(ppf.ARNA, 0.5)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            binned.append(pf.last_step_binned())
        lostrun[name] = {"step_ms_per_frame": ms, "binned": binned}
        pf.close()
    out["lost_object_arna"] = lostrun
    out["timing"] = "CUDA events around ppf_step (frame preparation and every kernel of the step)"
    return out


def run_ours(args):
    import torch
    import paper_1310_5045_gb300 as ppf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    n = args.n
    K, Wm = args.steps, args.warmup
    extra = 0 if args.no_schemes else len(SCHEME_ROWS) * (args.scheme_steps + 2)
    k_total = Wm + TIMED_RUNS * K + extra + (args.e2e_steps if not args.no_e2e else 0) + 2
    mv, params = make_workload(k_total, seed=0)
    model = ppf.Model(**params, seed=rank, filter_id=rank)
    frames = torch.from_numpy(mv.frames).to(dev)
    stream = torch.cuda.current_stream()
    pf = ppf.ParticleFilter(model, n, group_size=GROUP, stream=stream)
    scheme = ppf.SCHEMES[args.scheme]
    for k in range(1, Wm + 1):
        pf.step(frames[k - 1], k)
        pf.resample(scheme, args.alpha)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # TIMED_RUNS runs of exactly K frames each, on consecutive frames; each
    # run is bracketed by a barrier and a synchronisation, its time is the
    # slowest rank's, and the median run is reported
    pf.profile_enable(True, capacity=TIMED_RUNS * K + 8)
    clocks = ClockSampler(torch.cuda.current_device(), period_ms=50)
    runs_ms = []
    k0 = Wm + 1
    for _ in range(TIMED_RUNS):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t = timed_frames(pf, frames, k0, K, scheme, args.alpha, stream)
        torch.cuda.synchronize()
        runs_ms.append(max_over_ranks(t, dist, dev))
        k0 += K
    clk = clocks.stop()
    t_ms = statistics.median(runs_ms)
    prof = pf.profile_read()
    est = pf.estimate()
    kdone = k0 - 1
    value = job_rate(n, K, world, t_ms)

    step_ms = prof["step_ms"] / max(1, prof["timed_steps"])
    achieved = STEP_BYTES * n / (step_ms / 1e3) / 1e9
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))
    peak = float(peaks.get("hbm_gbs", 6800.0))
    traffic = None if STEP_TRAFFIC_PER_PARTICLE is None else STEP_TRAFFIC_PER_PARTICLE * n
    roofline = {"bound": "hbm", "kernel": "step_kernel<5> (propagate + likelihood + weight partials)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback",
                "bytes_per_particle": STEP_BYTES, "step_kernel_ms": step_ms,
                "traffic": traffic,
                "traffic_source": "ncu dram bytes at N=16M scaled by N (profiles/step_kernel_direct_spot512_n8m.md)",
                "phase_ms_per_step": {kk: prof[kk] / max(1, prof["timed_steps"]) for kk in
                                      ("prepare_ms", "step_ms", "finalize_ms", "resample_ms")}}
    # FP32 peak: FMA chains on every SM (scalar and packed two-lane), timed
    # with CUDA events, the SM clock sampled meanwhile
    fp32 = {}
    try:
        # about two seconds of launches, so that the clock sampler sees them
        pclk = ClockSampler(torch.cuda.current_device(), period_ms=50)
        t_end = time.perf_counter() + 2.0
        while time.perf_counter() < t_end:
            for name, packed in (("ffma", False), ("ffma2", True)):
                tf, ms = ppf.fp32_peak(packed=packed, repeats=20)
                if name not in fp32 or tf > fp32[name]["tflops"]:
                    fp32[name] = {"tflops": tf, "ms_per_launch": ms}
        fp32["clocks"] = pclk.stop()
        fp32_peak = max(fp32["ffma"]["tflops"], fp32["ffma2"]["tflops"])
        peak_src = ("measured: FMA chains on every SM, best of the scalar and packed two-lane forms, CUDA events "
                    "(ppf_fp32_peak)")
    except Exception as e:  # noqa: BLE001 - the derived figure is reported with its source
        fp32_peak = FP32_PEAK_DERIVED_TFLOPS
        peak_src = f"derived (152 SMs x 128 lanes x 2 x 2.07 GHz); measurement failed: {e}"
    tflops = STEP_FLOPS * n / (step_ms / 1e3) / 1e12
    tflops_px = STEP_FLOPS_PER_PIXEL_FORM * n / (step_ms / 1e3) / 1e12
    roofline_alu = {"bound": "alu", "kernel": "step_kernel<5>", "achieved": tflops, "peak": fp32_peak,
                    "unit": "TFLOP/s", "frac": tflops / fp32_peak, "flops_per_particle": STEP_FLOPS,
                    "per_pixel_form": {"flops_per_particle": STEP_FLOPS_PER_PIXEL_FORM, "achieved": tflops_px,
                                       "frac": tflops_px / fp32_peak},
                    "peak_source": peak_src, "fp32_measured": fp32,
                    "peak_derived": FP32_PEAK_DERIVED_TFLOPS}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
            "ms_per_step": t_ms / K, "timing": f"median of {TIMED_RUNS} runs of {K} frames (CUDA events)",
            "runs_ms_per_step": [r / K for r in runs_ms],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded Poisson spot movie, random-init particles)",
            "config": workload_desc(n, args.scheme), "roofline": roofline, "roofline_alu": roofline_alu,
            "clocks": clk,
            "gpu_launches": int(prof["launches"]),
            "last_estimate": {"mean": est.mean, "ess": est.ess, "log_evidence": est.log_evidence,
                              "truth": mv.truth[kdone - 1].tolist()}}

    # end to end through the C ABI with host frames (pinned), every frame's
    # estimate read back (queued copies into page-locked slots, decoded on
    # the host after the last frame)
    if not args.no_e2e:
        ke = args.e2e_steps
        host = torch.from_numpy(mv.frames[kdone:kdone + ke]).pin_memory()  # the frames right after the timed ones
        slots = torch.empty((ke, ppf.Estimate.nbytes()), dtype=torch.uint8).pin_memory()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        pf.profile_enable(True, capacity=ke + 8)
        t0 = time.perf_counter()
        for i in range(ke):
            pf.step_host(host[i], kdone + 1 + i)
            pf.resample(scheme, args.alpha)
            pf.estimate_async(slots[i])
        torch.cuda.synchronize()
        e2e_est = [ppf.Estimate.from_buffer(slots[i]) for i in range(ke)]
        dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
        pr = pf.profile_read()
        line["e2e"] = {"value": job_rate(n, ke, world, 1e3 * dt), "unit": UNIT, "steps": ke,
                       "h2d_bytes_per_step": pr["h2d_bytes"] // ke, "d2h_bytes_per_step": pr["d2h_bytes"] // ke,
                       "timing": "host wall clock around ppf_step_host + ppf_resample + ppf_estimate_async per "
                                 "frame and the final synchronisation and decoding of every frame's estimate, on "
                                 "the frames that follow the timed ones",
                       "last_frame": e2e_est[-1].frame}
        kdone += ke

    # every allocation / routing scheme of Sec. 3-4 on the same workload
    if not args.no_schemes:
        sch = {}
        k = kdone + 1
        # every row starts from balanced groups except the LGS rows, which
        # unbalance them themselves (they run last so that no other row
        # inherits their layout)
        for name, alpha in SCHEME_ROWS:
            sid = ppf.SCHEMES[name]
            for _ in range(2):
                pf.step(frames[k - 1], k)
                pf.resample(sid, alpha)
                k += 1
            tm = timed_frames(pf, frames, k, args.scheme_steps, sid, alpha, stream)
            k += args.scheme_steps
            e = pf.estimate()
            key = name if name != "rna" else f"rna_{alpha}"
            sch[key] = {"value": n * args.scheme_steps / (tm / 1e3), "ms_per_step": tm / args.scheme_steps,
                        "links": e.links, "moved": e.moved, "max_group": e.max_group, "min_group": e.min_group}
        line["schemes"] = sch
        kdone = k - 1

    # the spread regime (Sec. 6.3's input-space decomposition): the prior draw
    # of frame 1 covers the whole frame, and a lost object leaves the weights
    # flat; each likelihood path on them
    if not args.no_spread:
        line["spread"] = spread_ab(ppf, params, rank, n, stream, args)

    # pcSIR (Sec. 6): the same workload with the piecewise constant likelihood
    # (one lookup per particle in the per-frame map of cell-centre patch sums)
    if not args.no_pcsir:
        ppc = ppf.ParticleFilter(ppf.Model(**params, seed=rank, filter_id=rank, likelihood=1), n,
                                 group_size=GROUP, stream=stream)
        for k in range(1, Wm + 1):
            ppc.step(frames[k - 1], k)
            ppc.resample(scheme, args.alpha)
        torch.cuda.synchronize()
        ppc.profile_enable(True, capacity=K + 8)
        tpc = timed_frames(ppc, frames, Wm + 1, K, scheme, args.alpha, stream)
        prc = ppc.profile_read()
        epc = ppc.estimate()
        line["pcsir"] = {"workload": "the same frames and N with the piecewise constant likelihood (pcSIR)",
                         "value": n * K / (tpc / 1e3), "ms_per_step": tpc / K,
                         "step_ms": prc["step_ms"] / max(1, prc["timed_steps"]),
                         "prepare_ms": prc["prepare_ms"] / max(1, prc["timed_steps"]),
                         "resample_ms": prc["resample_ms"] / max(1, prc["timed_steps"]),
                         "last_mean_xy": list(epc.mean[:2]), "truth_xy": mv.truth[Wm + K - 1][:2].tolist()}
        ppc.close()
        del ppc

    # batched filters: 4096 filters, N_f log-uniform in [256, 65536], 64^2 frames
    if not args.no_batch:
        import synth
        Kb = 2 + 3 * args.batch_steps
        mb = synth.make_movie_batch(F=args.batch_filters, W=64, H=64, K=Kb, n_range=(256, 65536), seed=0)
        bmodels = [ppf.Model(width=64, height=64, patch_radius=5, psf_sigma=float(mb.sigma[f]),
                             amplitude=float(mb.amplitude[f]), background=10.0, sigma_xi=math.sqrt(10.0),
                             sigma_m=0.5, sigma_v=0.1, sigma_I=1.0, seed=rank, filter_id=f)
                   for f in range(args.batch_filters)]
        bfr = torch.from_numpy(mb.frames).to(dev)
        bres = {}
        bf = ppf.BatchFilter(bmodels, mb.n_particles, stream=stream)
        bf.run(bfr[:2], 1, use_graph=True, estimates=False)
        # tune the launch shape on the third frame, once the clouds have
        # concentrated (the prior draw of frame 1 reads the frames very differently)
        cfg = None if args.no_autotune else bf.autotune(bfr[2], 3)
        k0 = 3
        for mode in ("graph", "launches", "graph"):  # same launch shape; the graph twice (first and last)
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            bf.run(bfr[k0 - 1:k0 - 1 + args.batch_steps], k0, use_graph=(mode == "graph"), estimates=False)
            ev1.record(stream)
            ev1.synchronize()
            dt = ev0.elapsed_time(ev1) / 1e3
            k0 += args.batch_steps
            r = {"particle_steps_per_sec": bf.ntot * args.batch_steps / dt, "ms_per_frame": 1e3 * dt / args.batch_steps}
            if mode not in bres or r["ms_per_frame"] < bres[mode]["ms_per_frame"]:
                bres[mode] = r
        bres["graph"]["autotuned"] = cfg if cfg else "off (default shape)"
        ntot = bf.ntot
        bf.close()
        line["batched"] = {"workload": f"{args.batch_filters} filters, N_f log-uniform in [256, 65536] "
                                       f"(total {ntot:,}), 64x64 frames, 11x11 patch, systematic per filter",
                           "filters": args.batch_filters, "particles": ntot, "frames_timed": args.batch_steps,
                           "timing": "CUDA events around one ppf_batch_run of the timed frames (the graph: best of "
                                     "two runs), autotuned launch shape for both", **bres,
                           "vs_plain_fp32_path": bres["graph"]["particle_steps_per_sec"] / value}
        del bfr

    # reduced-precision frames: BF16 / FP16 against the FP32 path, per frame in
    # lockstep (both start every frame from the FP32 run's particles)
    if not args.no_precision:
        prec = {}
        pn = args.precision_n
        gain = torch.from_numpy(mv.frames[: args.precision_frames + 1]).to(dev) * 1.37 + 0.29
        base = ppf.ParticleFilter(ppf.Model(**params, seed=rank), pn, group_size=GROUP, stream=stream)
        others = {}
        for name, dt_, code in (("bf16", torch.bfloat16, ppf.BF16), ("fp16", torch.float16, ppf.F16)):
            others[name] = (ppf.ParticleFilter(ppf.Model(**params, seed=rank, frame_dtype=code), pn, group_size=GROUP,
                                               stream=stream), gain.to(dt_).contiguous())
        errs = {name: {"mean_rel": 0.0, "log_evidence_rel": 0.0} for name in others}
        for k in range(1, args.precision_frames + 1):
            st, an, lp = base.get_particles(state=True, anc=True, lw_prev=True)
            for name, (pf2, fr2) in others.items():
                pf2.set_particles(st, an if k > 1 else None, lp if k > 1 else None)
            base.step(gain[k - 1].contiguous(), k)
            e32 = base.estimate()
            for name, (pf2, fr2) in others.items():
                pf2.step(fr2[k - 1], k)
                e2 = pf2.estimate()
                scales = np.array([W, H, 1.0, 1.0, params["amplitude"]])
                m = np.max(np.abs(np.array(e2.mean) - np.array(e32.mean)) / np.maximum(np.abs(e32.mean), scales))
                errs[name]["mean_rel"] = max(errs[name]["mean_rel"], float(m))
                errs[name]["log_evidence_rel"] = max(errs[name]["log_evidence_rel"],
                                                     abs(e2.log_evidence - e32.log_evidence) / abs(e32.log_evidence))
            base.resample(ppf.SYSTEMATIC)
        for name, (pf2, fr2) in others.items():
            # throughput of the reduced-precision path on the same frames
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            pf2.resample(ppf.SYSTEMATIC)
            e0.record(stream)
            for k in range(1, args.precision_frames + 1):
                pf2.step(fr2[k - 1], 100 + k)
                pf2.resample(ppf.SYSTEMATIC)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / args.precision_frames
            prec[name] = {"max_rel_err_mean_vs_fp32": errs[name]["mean_rel"],
                          "max_rel_err_log_evidence_vs_fp32": errs[name]["log_evidence_rel"],
                          "ms_per_frame": ms, "particle_steps_per_sec": pn / (ms / 1e3)}
            pf2.close()
        base.close()
        line["precision"] = {"workload": f"N={pn:,}, the 512x512 movie scaled by 1.37 and offset by 0.29 "
                                         "(non-integer counts, so BF16/FP16 storage rounds them)",
                             "frames": args.precision_frames, **prec,
                             "note": "integer photon counts <= 256 are exact in BF16 (<= 2048 in FP16): on the "
                                     "unscaled movie the reduced-precision paths reproduce FP32 bit for bit",
                             "vs_fp64_oracle": "per frame, N=2^20 and 38M, five seeds: tests/test_gpu_precision.py"}

    # gradient of the log marginal likelihood: N = 2^20, 50 frames of 256^2
    if not args.no_grad:
        import synth
        gmv, gp = synth.preset("spot256_k50", seed=1)
        gmodel = ppf.Model(width=256, height=256, patch_radius=4, psf_sigma=1.5, amplitude=50.0, background=10.0,
                           sigma_xi=math.sqrt(10.0), sigma_m=0.5, sigma_v=0.1, sigma_I=0.0, seed=rank)
        gfr = torch.from_numpy(gmv.frames).to(dev)
        gpf = ppf.ParticleFilter(gmodel, gp["N"], group_size=GROUP, stream=stream)
        gpf.loglik_grad(gfr)
        torch.cuda.synchronize()
        reps = args.grad_evals
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            Lg, gg = gpf.loglik_grad(gfr)
        e1.record(stream)
        e1.synchronize()
        tg = e0.elapsed_time(e1) / reps
        K5 = gfr.shape[0]
        line["grad"] = {"workload": f"spot256: 256x256 frames, K={K5}, N={gp['N']}, 9x9 patch, I0 = A, "
                                    "systematic resampling (stop-gradient)",
                        "grad_evals_per_sec": 1e3 / tg, "ms_per_eval": tg,
                        "particle_steps_per_sec": gp["N"] * K5 / (tg / 1e3),
                        "loglik": Lg, "grad": {"psf_sigma": gg[0], "amplitude": gg[1], "background": gg[2],
                                               "sigma_m": gg[3]},
                        }
        gpf.close()

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(params, mv.frames, args.cpu_n, args.cpu_frames)
    pf.close()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


PROFILE_CASES = ("step", "rpa_gs", "rpa_sgs", "rpa_lgs", "rpa2_gs", "rpa2_lgs", "rna", "arna", "binned", "pcsir", "grad",
                 "batch")


def run_profile_case(args):
    """A small run of one kernel family for an ncu capture (no JSON line): the
    spot512 workload at --n particles, 6 frames (the first two with systematic
    resampling to concentrate the cloud, then the case's scheme); "binned"
    forces the binned likelihood on the prior draw of frame 1; "grad" runs
    the gradient over 5 frames of 256^2 at --n; "batch" runs 512 filters."""
    import torch
    import paper_1310_5045_gb300 as ppf
    import synth
    case, n = args.profile, args.n
    dev = torch.device("cuda", torch.cuda.current_device())
    if case == "grad":
        gmv, _ = synth.preset("spot256_k50", seed=1, K=5)
        gm = ppf.Model(width=256, height=256, patch_radius=4, psf_sigma=1.5, amplitude=50.0, background=10.0,
                       sigma_xi=math.sqrt(10.0), sigma_m=0.5, sigma_v=0.1, sigma_I=0.0, seed=0)
        pf = ppf.ParticleFilter(gm, n, group_size=GROUP)
        fr = torch.from_numpy(gmv.frames).to(dev)
        for _ in range(2):
            pf.loglik_grad(fr)
        pf.close()
        return 0
    if case == "batch":
        mb = synth.make_movie_batch(F=512, W=64, H=64, K=6, n_range=(256, 65536), seed=0)
        models = [ppf.Model(width=64, height=64, patch_radius=5, psf_sigma=float(mb.sigma[f]),
                            amplitude=float(mb.amplitude[f]), background=10.0, sigma_xi=math.sqrt(10.0),
                            sigma_m=0.5, sigma_v=0.1, sigma_I=1.0, seed=0, filter_id=f) for f in range(512)]
        bf = ppf.BatchFilter(models, mb.n_particles)
        bf.run(torch.from_numpy(mb.frames).to(dev), 1, use_graph=False, estimates=False)
        torch.cuda.synchronize()
        bf.close()
        return 0
    mv, params = make_workload(8, seed=0)
    fr = torch.from_numpy(mv.frames).to(dev)
    model = ppf.Model(**params, seed=0, likelihood=1 if case == "pcsir" else 0)
    pf = ppf.ParticleFilter(model, n, group_size=GROUP)
    pf.set_likelihood_path(ppf.PATH_BINNED if case == "binned" else
                           (ppf.PATH_AUTO if case == "pcsir" else ppf.PATH_DIRECT))
    scheme = ppf.SCHEMES["systematic" if case in ("step", "binned", "pcsir") else case]
    for k in range(1, 7):
        pf.step(fr[k - 1], k)
        pf.resample(ppf.SYSTEMATIC if k <= 2 else scheme, 0.5)
    torch.cuda.synchronize()
    pf.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_FULL)
    ap.add_argument("--scheme", default="systematic", choices=sorted(["systematic", "rpa_gs", "rpa_sgs",
                                                                      "rpa_lgs", "rna", "rpa2_gs", "rpa2_sgs",
                                                                      "rpa2_lgs", "arna"]))
    ap.add_argument("--alpha", type=float, default=0.1)
    ap.add_argument("--scheme-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--cpu-n", type=int, default=N_FULL)
    ap.add_argument("--cpu-frames", type=int, default=2)
    ap.add_argument("--ref-n", type=int, default=1 << 21)
    ap.add_argument("--no-schemes", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-pcsir", action="store_true")
    ap.add_argument("--no-spread", action="store_true")
    ap.add_argument("--batch-filters", type=int, default=4096)
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--no-autotune", action="store_true", help="batched stage: keep the default launch shape")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--precision-n", type=int, default=N_FULL)
    ap.add_argument("--precision-frames", type=int, default=5)
    ap.add_argument("--grad-evals", type=int, default=3)
    ap.add_argument("--profile", choices=PROFILE_CASES, default=None,
                    help="run a small case of one kernel family for an ncu capture (prints no JSON line)")
    args = ap.parse_args()
    if args.profile:
        return run_profile_case(args)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
