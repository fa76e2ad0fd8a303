"""Parity at the full benchmark size: N = 38,000,000 particles, 512 x 512
frames, 11 x 11 patch, groups of 4096 -- the launch configuration bench.py
times.  Propagation and likelihood are checked on sampled slots that the
oracle computes one by one; normalisation, estimate and log-evidence by the
oracle's FP64 summary over all particles (same log-weight inputs, exact bound
as in gpu_common); the ancestors and group offsets bit-exactly for systematic,
RPA-LGS, RPA-SGS, two-stage RPA-LGS, RNA, two-stage RPA-GS and ARNA
resampling (the oracle resamples all 38 M weights).  Above 16384 tiles
(N > 67,108,864) the one-block tile scan walks the tile sums in rounds
instead of shared memory; a filter of 67,112,961 particles checks that path
the same way."""
import math

import numpy as np
import pytest

import oracle as orc
import synth

pytestmark = pytest.mark.gpu

N_FULL = 38_000_000


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 8 * 2**30:
        pytest.skip("needs ~8 GB of free device memory")
    import paper_1310_5045_gb300 as ppf
    from gpu_common import paired_models
    mv, p = synth.preset("spot512_k50", seed=0, K=7)
    gm, om = paired_models(ppf, width=512, height=512, patch_radius=5, psf_sigma=float(p["sigma"]),
                           amplitude=float(p["amplitude"]), seed=0)
    frames = torch.from_numpy(mv.frames).cuda()
    pf = ppf.ParticleFilter(gm, N_FULL, group_size=4096)
    yield ppf, pf, gm, om, mv, frames
    pf.close()


def one_frame(ppf, pf, gm, om, mv, frames, k, scheme, alpha=0.1, n_sample=20000):
    import torch
    N_FULL = pf.n
    rng = np.random.default_rng(k)
    st0, anc0, lwp0 = pf.get_particles(state=True, anc=True, lw_prev=True)
    goff0 = pf.groups()
    pf.step(frames[k - 1], k)
    st1, _, _ = pf.get_particles()
    est = pf.estimate()
    slots = np.sort(rng.choice(N_FULL, size=n_sample, replace=False))
    sl = torch.from_numpy(slots).cuda()
    anc_s = anc0[sl].long()
    parents = st0[:5, anc_s].double().cpu().numpy()
    S = st1[:, sl].double().cpu().numpy()
    lp = lwp0[sl].double().cpu().numpy()
    # S1 on sampled slots
    ref = orc.propagate_slots(om, k, slots, parents)
    scale = np.abs(parents).copy()
    scale[0] += np.abs(parents[2])
    scale[1] += np.abs(parents[3])
    sig = np.array([gm.sigma_m, gm.sigma_m, gm.sigma_v, gm.sigma_v, gm.sigma_I])[:, None]
    assert np.all(np.abs(S[:5] - ref) <= 2e-6 * (scale + 6 * sig + 1.0))
    # S3 on the same slots
    fr = mv.frames[k - 1].astype(np.float64)
    l_ref = orc.loglik_many(om, fr, S[0], S[1], S[4])
    tol = 1e-5 * np.maximum(1.0, np.abs(l_ref)) + 1e-6 * S[4] ** 2 * 121 / gm.sigma_xi ** 2
    lw_ref = lp + l_ref
    assert np.all(np.abs(S[5] - lw_ref) <= tol + 4 * np.spacing(np.abs(lw_ref).astype(np.float32)))
    # S4/S5 over all particles from the GPU's float32 state and log-weights
    full = st1.double().cpu().numpy()
    so = orc.summary(full, lwp0.double().cpu().numpy())
    scales = np.array([gm.width, gm.height, 1.0, 1.0, gm.amplitude])
    assert np.all(np.abs(np.asarray(est.mean) - so["mean"]) <= 1e-4 * np.maximum(np.abs(so["mean"]), scales))
    assert abs(est.log_evidence - so["log_evidence"]) <= 1e-5 * max(1.0, abs(so["log_evidence"]))
    assert abs(est.ess - so["ess"]) <= 1e-4 * so["ess"]
    # S6-S8 bit-exact from the same float32 log-weights
    lwf = st1[5].cpu().numpy()
    del full
    ring0 = pf.ring() if scheme == orc.ARNA else None
    pf.resample(scheme, alpha)
    _, anc1, lwp1 = pf.get_particles(state=False, anc=True, lw_prev=True)
    e2 = pf.estimate()
    if scheme == orc.ARNA:
        lost = bool(e2.status_flags & 32)
        assert lost == (so["log_evidence"] < 0.0)
        rc, anc_ref, lwr_ref, goff_ref, stats, ring_ref = orc.resample_arna(
            om, N_FULL, k, goff0, lwf, lost, ring0, lw_sum=lwf.astype(np.float64), alpha=float(np.float32(alpha)))
        assert np.array_equal(pf.ring(), ring_ref)
        stats = stats[:4]
    else:
        rc, anc_ref, lwr_ref, goff_ref, stats = orc.resample(om, scheme, N_FULL, k, goff0, lwf,
                                                             lwf.astype(np.float64), alpha)
    assert rc == 0
    a1 = anc1.cpu().numpy()
    assert np.array_equal(a1, anc_ref), int(np.sum(a1 != anc_ref))
    assert np.array_equal(pf.groups(), goff_ref)
    if scheme in (orc.RNA, orc.ARNA):
        l1 = lwp1.double().cpu().numpy()
        assert np.all(np.abs(l1 - lwr_ref) <= 1e-5 * np.maximum(1.0, np.abs(lwr_ref)))
    assert (e2.links, e2.moved, e2.max_group, e2.min_group) == tuple(int(v) for v in stats)
    return est


def test_full_size_frames(setup):
    ppf, pf, gm, om, mv, frames = setup
    # LGS leaves unequal groups: the one-stage SGS and two-stage GS frames
    # after it route their kept tickets from tiles crossed by unequal groups
    one_frame(ppf, pf, gm, om, mv, frames, 1, orc.SYSTEMATIC)
    one_frame(ppf, pf, gm, om, mv, frames, 2, orc.RPA_LGS)
    one_frame(ppf, pf, gm, om, mv, frames, 3, orc.RPA_SGS)
    one_frame(ppf, pf, gm, om, mv, frames, 4, orc.RPA2_LGS)
    est = one_frame(ppf, pf, gm, om, mv, frames, 5, orc.RNA, alpha=0.1)
    assert math.isfinite(est.log_evidence)
    est = one_frame(ppf, pf, gm, om, mv, frames, 6, orc.RPA2_GS)
    assert math.isfinite(est.log_evidence)
    est = one_frame(ppf, pf, gm, om, mv, frames, 7, orc.ARNA, alpha=0.5)
    assert math.isfinite(est.log_evidence)


# 16384 tiles of 4096 and a ragged tile of 4097 more: the tile scan walks the
# 16386 tile sums in rounds (more than its shared memory holds)
N_ROUNDS = 16384 * 4096 + 4097


def test_tile_scan_in_rounds_above_16384_tiles():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 16 * 2**30:
        pytest.skip("needs ~16 GB of free device memory")
    import paper_1310_5045_gb300 as ppf
    from gpu_common import paired_models
    mv, p = synth.preset("spot512_k50", seed=1, K=3)
    gm, om = paired_models(ppf, width=512, height=512, patch_radius=5, psf_sigma=float(p["sigma"]),
                           amplitude=float(p["amplitude"]), seed=1)
    frames = torch.from_numpy(mv.frames).cuda()
    # groups of 8192: 8193 groups, within the RPA schedule's 16384
    pf = ppf.ParticleFilter(gm, N_ROUNDS, group_size=8192)
    try:
        # frame 1 from the prior (the spread cloud takes the binned path),
        # then a routed RPA draw and an RNA draw over the concentrated cloud
        one_frame(ppf, pf, gm, om, mv, frames, 1, orc.SYSTEMATIC)
        assert pf.last_step_binned()
        one_frame(ppf, pf, gm, om, mv, frames, 2, orc.RPA_SGS)
        est = one_frame(ppf, pf, gm, om, mv, frames, 3, orc.RNA, alpha=0.1)
        assert math.isfinite(est.log_evidence)
    finally:
        pf.close()
