"""Batched filters (ppf_batch_*): every filter against the FP64 oracle in
lockstep (same tolerances as tests/gpu_common.py, bit-exact ancestors),
bitwise equality with single-filter contexts, CUDA-graph runs identical to
plain launches, and autotuned launch shapes that leave the results unchanged."""
import math

import numpy as np
import pytest

import oracle as orc
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1310_5045_gb300 as p
    p.load()
    return p


def make(ppf, F, ns, K=4, seed=0, W=48, sigma_xi2=10.0):
    import torch
    from gpu_common import f32
    mb = synth.make_movie_batch(F=F, W=W, H=W, K=K, n_range=(256, 1024), seed=seed)
    gms, oms = [], []
    for f in range(F):
        kw = dict(width=W, height=W, patch_radius=4, psf_sigma=f32(mb.sigma[f]), amplitude=f32(mb.amplitude[f]),
                  background=10.0, sigma_xi=f32(math.sqrt(sigma_xi2)), sigma_m=0.5, sigma_v=0.1, sigma_I=1.0,
                  v0_max=1.0, seed=seed, filter_id=f)
        gms.append(ppf.Model(**kw))
        oms.append(orc.Model(**kw))
    frames = torch.from_numpy(np.ascontiguousarray(mb.frames)).cuda()   # (K, F, H, W)
    return mb, gms, oms, frames


def test_batch_lockstep_against_oracle(ppf):
    F = 9
    ns = [1, 7, 300, 4095, 4096, 4097, 9000, 250, 2]
    mb, gms, oms, frames = make(ppf, F, ns)
    bf = ppf.BatchFilter(gms, ns)
    off = bf.offsets
    for k in range(1, 4):
        st0, anc0 = bf.get_particles(state=True, anc=(k > 1))
        st0 = st0.double().cpu().numpy()
        a0 = anc0.cpu().numpy() if anc0 is not None else np.arange(bf.ntot, dtype=np.int32)
        bf.step(frames[k - 1], k)
        est = bf.estimates()
        st1, _ = bf.get_particles()
        S = st1.double().cpu().numpy()
        bf.resample(k)
        _, anc1 = bf.get_particles(state=False, anc=True)
        a1 = anc1.cpu().numpy()
        for f in range(F):
            lo, hi = off[f], off[f + 1]
            n = hi - lo
            par = st0[:, lo:hi]
            anc = a0[lo:hi] - lo
            ref = orc.propagate(oms[f], k, par, anc, np.zeros(n) if k > 1 else par[5])
            assert np.all(np.abs(S[:5, lo:hi] - ref[:5]) <= 2e-6 * (np.abs(ref[:5]) + 10.0)), f
            fr = mb.frames[k - 1, f].astype(np.float64)
            lp = np.zeros(n) if k > 1 else par[5][anc]
            l_ref = orc.loglik_many(oms[f], fr, S[0, lo:hi], S[1, lo:hi], S[4, lo:hi])
            tol = 1e-5 * np.maximum(1.0, np.abs(l_ref)) + 1e-6 * S[4, lo:hi] ** 2 * 81 / 10.0
            assert np.all(np.abs(S[5, lo:hi] - (lp + l_ref)) <= tol + 1e-6 * np.abs(l_ref)), f
            so_st = S[:, lo:hi].copy()
            so_st[5] = lp + l_ref
            so = orc.summary(so_st, lp)
            scale = np.array([48.0, 48.0, 1.0, 1.0, gms[f].amplitude])
            assert np.all(np.abs(est[f]["mean"] - so["mean"]) <= 1e-4 * np.maximum(np.abs(so["mean"]), scale)), f
            assert abs(est[f]["log_evidence"] - so["log_evidence"]) <= 1e-5 * max(1.0, abs(so["log_evidence"]))
            lwf = st1[5, lo:hi].cpu().numpy()
            rc, want, _, _, _ = orc.resample(oms[f], orc.SYSTEMATIC, n, k, np.array([0, n]), lwf)
            assert rc == 0 and np.array_equal(a1[lo:hi] - lo, want), f
    bf.close()


def test_batch_equals_single_filter_contexts(ppf):
    F = 5
    ns = [513, 64, 5000, 1, 2048]
    mb, gms, oms, frames = make(ppf, F, ns, seed=3)
    bf = ppf.BatchFilter(gms, ns)
    singles = [ppf.ParticleFilter(gms[f], ns[f], group_size=ns[f]) for f in range(F)]
    for k in range(1, 4):
        bf.step(frames[k - 1], k)
        for f in range(F):
            singles[f].step(frames[k - 1, f].contiguous(), k)
        sb, _ = bf.get_particles()
        for f in range(F):
            s1, _, _ = singles[f].get_particles()
            assert np.array_equal(sb[:, bf.offsets[f]:bf.offsets[f + 1]].cpu().numpy(), s1.cpu().numpy()), (k, f)
        bf.resample(k)
        _, ab = bf.get_particles(state=False, anc=True)
        for f in range(F):
            singles[f].resample(ppf.SYSTEMATIC)
            _, a1, _ = singles[f].get_particles(state=False, anc=True)
            assert np.array_equal(ab[bf.offsets[f]:bf.offsets[f + 1]].cpu().numpy() - bf.offsets[f],
                                  a1.cpu().numpy()), (k, f)
    for s in singles:
        s.close()
    bf.close()


def test_batch_ess_test_equals_single_filter_contexts(ppf):
    """Alg. 1's N_eff test per filter: the batch with fraction 0.3 against
    single-filter contexts resampling only while N_eff < 0.3 n_f (both sides
    decide from their own N_eff, so a filter is followed only while its N_eff
    is not within 1e-4 of the threshold)."""
    F = 6
    ns = [513, 64, 5000, 3, 2048, 900]
    K = 8
    mb, gms, oms, frames = make(ppf, F, ns, K=K, seed=4, sigma_xi2=2000.0)
    bf = ppf.BatchFilter(gms, ns)
    bf.set_ess_threshold(0.3)
    singles = [ppf.ParticleFilter(gms[f], ns[f], group_size=ns[f]) for f in range(F)]
    live = [True] * F
    kept_seen = resampled_seen = 0
    for k in range(1, K + 1):
        bf.step(frames[k - 1], k)
        for f in range(F):
            singles[f].step(frames[k - 1, f].contiguous(), k)
        sb, _ = bf.get_particles()
        for f in range(F):
            if live[f]:
                s1, _, _ = singles[f].get_particles()
                assert np.array_equal(sb[:, bf.offsets[f]:bf.offsets[f + 1]].cpu().numpy(), s1.cpu().numpy()), (k, f)
        bf.resample(k)
        _, ab = bf.get_particles(state=False, anc=True)
        for f in range(F):
            thr = 0.3 * ns[f]
            ess = singles[f].estimate().ess
            singles[f].resample(ppf.SYSTEMATIC, ess_threshold=thr)
            if abs(ess - thr) <= 1e-4 * thr:
                live[f] = False
            if not live[f]:
                continue
            if ess >= thr:
                kept_seen += 1
            else:
                resampled_seen += 1
            _, a1, _ = singles[f].get_particles(state=False, anc=True)
            assert np.array_equal(ab[bf.offsets[f]:bf.offsets[f + 1]].cpu().numpy() - bf.offsets[f],
                                  a1.cpu().numpy()), (k, f)
    assert kept_seen > 0 and resampled_seen > 0, (kept_seen, resampled_seen)
    for s in singles:
        s.close()
    bf.close()


def test_graph_run_matches_plain_launches_and_autotune(ppf):
    import torch
    F = 40
    rng = np.random.default_rng(1)
    ns = [int(v) for v in np.floor(np.exp(rng.uniform(np.log(256), np.log(6000), F)))]
    mb, gms, oms, frames = make(ppf, F, ns, K=5, seed=5)
    a = ppf.BatchFilter(gms, ns)
    b = ppf.BatchFilter(gms, ns)
    cfg = b.autotune(frames[0], 1)
    assert cfg["unit"] in (512, 1024, 2048, 4096) and cfg["block"] in (128, 256, 512)
    # two runs: the second replays the graph cached by the first, from the next frame
    a.run(frames[:2], 1, use_graph=False)
    b.run(frames[:2], 1, use_graph=True)
    ea = a.run(frames[2:], 3, use_graph=False)
    eb = b.run(frames[2:], 3, use_graph=True)
    sa, aa = a.get_particles(anc=True)
    sb, ab = b.get_particles(anc=True)
    assert torch.equal(sa, sb) and torch.equal(aa, ab)
    # a different work-unit size groups the float32 partial sums differently:
    # the estimates agree to the summation-order error
    assert np.allclose(ea["mean"], eb["mean"], rtol=1e-5, atol=1e-5)
    assert np.allclose(ea["log_evidence"], eb["log_evidence"], rtol=1e-6)
    a.close()
    b.close()


def test_step_api_matches_run(ppf):
    import torch
    F = 6
    ns = [100, 4097, 7, 3000, 1, 512]
    mb, gms, oms, frames = make(ppf, F, ns, K=3, seed=9)
    a = ppf.BatchFilter(gms, ns)
    b = ppf.BatchFilter(gms, ns)
    for k in range(1, 4):
        a.step(frames[k - 1], k)
        a.resample(k)
    b.run(frames, 1, use_graph=True)
    sa, aa = a.get_particles(anc=True)
    sb, ab = b.get_particles(anc=True)
    assert torch.equal(sa, sb) and torch.equal(aa, ab)
    with pytest.raises(ppf.PPFError):
        a.resample(3)  # no step since the last resample
    a.close()
    b.close()


def test_batch_full_size_sampled_filters(ppf):
    """The batched workload in full, in the benchmark's launch configuration:
    4096 filters, N_f log-uniform in [256, 65536] (about 49 M particles in
    all), 64 x 64 frames, 11 x 11 patch, 30 frames, the launch shape
    autotuned on the third frame.  Every frame, a sample of filters (the
    largest, the smallest and ten drawn at random) is checked against the
    oracle in lockstep: propagation, likelihood, estimate and log-evidence
    within gpu_common's tolerances, ancestors bit-exact."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < 8 * 2**30:
        pytest.skip("needs ~8 GB of free device memory")
    from gpu_common import MEAN_RTOL, LOGEV_RTOL, f32, loglik_tol
    F, K, Wd = 4096, 30, 64
    mb = synth.make_movie_batch(F=F, W=Wd, H=Wd, K=K, n_range=(256, 65536), seed=0)
    gms, oms = [], []
    for f in range(F):
        kw = dict(width=Wd, height=Wd, patch_radius=5, psf_sigma=f32(mb.sigma[f]), amplitude=f32(mb.amplitude[f]),
                  background=10.0, sigma_xi=f32(math.sqrt(10.0)), sigma_m=0.5, sigma_v=0.1, sigma_I=1.0,
                  v0_max=1.0, seed=0, filter_id=f)
        gms.append(ppf.Model(**kw))
        oms.append(orc.Model(**kw))
    frames = torch.from_numpy(np.ascontiguousarray(mb.frames)).cuda()
    ns = mb.n_particles
    bf = ppf.BatchFilter(gms, ns)
    off = bf.offsets
    assert off[-1] == int(ns.sum()) > 40_000_000
    rng = np.random.default_rng(5)
    orc.set_threads(0)
    for k in range(1, K + 1):
        if k == 3:
            bf.autotune(frames[2], 3)
        pick = np.unique(np.concatenate([[int(np.argmax(ns)), int(np.argmin(ns))], rng.choice(F, 10, replace=False)]))
        st0, anc0 = bf.get_particles(state=True, anc=(k > 1))
        sl0 = {f: st0[:, off[f]:off[f + 1]].double().cpu().numpy() for f in pick}
        a0 = {f: (anc0[off[f]:off[f + 1]].cpu().numpy() - off[f]) if anc0 is not None
              else np.arange(off[f + 1] - off[f], dtype=np.int32) for f in pick}
        del st0, anc0
        bf.step(frames[k - 1], k)
        est = bf.estimates()
        st1, _ = bf.get_particles()
        sl1 = {f: st1[:, off[f]:off[f + 1]].double().cpu().numpy() for f in pick}
        lwf = {f: st1[5, off[f]:off[f + 1]].cpu().numpy() for f in pick}
        del st1
        bf.resample(k)
        _, anc1 = bf.get_particles(state=False, anc=True)
        a1 = {f: anc1[off[f]:off[f + 1]].cpu().numpy() - off[f] for f in pick}
        del anc1
        for f in pick:
            n = off[f + 1] - off[f]
            par, S, om = sl0[f], sl1[f], oms[f]
            lp = np.zeros(n) if k > 1 else par[5][a0[f]]
            ref = orc.propagate(om, k, par, a0[f], lp)
            pp = par[:, a0[f]]
            scale = np.abs(pp[:5]).copy()
            scale[0] += np.abs(pp[2])
            scale[1] += np.abs(pp[3])
            sig = np.array([0.5, 0.5, f32(0.1), f32(0.1), 1.0])[:, None]
            assert np.all(np.abs(S[:5] - ref[:5]) <= 2e-6 * (scale + 6 * sig + 1.0)), (k, f)
            l_ref = orc.loglik_many(om, mb.frames[k - 1, f].astype(np.float64), S[0], S[1], S[4])
            lw_ref = lp + l_ref
            tol = loglik_tol(l_ref, S[4], 5, om.sigma_xi) + 4 * np.spacing(np.abs(lw_ref).astype(np.float32))
            assert np.all(np.abs(S[5] - lw_ref) <= tol), (k, f)
            so_st = S.copy()
            so_st[5] = lw_ref
            so = orc.summary(so_st, lp)
            sc = np.array([Wd, Wd, 1.0, 1.0, om.amplitude])
            assert np.all(np.abs(est[f]["mean"] - so["mean"]) <= MEAN_RTOL * np.maximum(np.abs(so["mean"]), sc)), (k, f)
            assert abs(est[f]["log_evidence"] - so["log_evidence"]) <= LOGEV_RTOL * max(1.0, abs(so["log_evidence"]))
            rc, want, _, _, _ = orc.resample(om, orc.SYSTEMATIC, n, k, np.array([0, n]), lwf[f])
            assert rc == 0 and np.array_equal(a1[f], want), (k, f)
    bf.close()
