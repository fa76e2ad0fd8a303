"""Shared helpers of the GPU parity tests: paired models (identical float32
parameters on both sides) and the per-frame lockstep comparison.

Tolerances (derived from the float32 arithmetic of the kernels):
  * propagation: x' = x + vx + s*e in float32 vs FP64 on identical inputs and
    Philox words: two roundings of |x| + |vx| plus the few-ulp error of the
    float32 log / sqrt / sincospi in e, so |d| <= 2e-6 (|x| + |v| + 6 s + 1).
  * likelihood: l = I0 (B - I0 C / 2) / sigma_xi^2 with B, C sums of at most
    (2r+1)^2 float32 products whose own error is a few ulp, so
    |d| <= 1e-5 max(1, |l|) + 1e-6 I0^2 (2r+1)^2 / sigma_xi^2.
  * posterior mean: 1e-4 relative to max(|ref|, scale), scale = W, H, 1, 1, A.
  * log-evidence: 1e-5 relative (to max(|ref|, 1)).
  * N_eff = (sum w)^2 / sum w^2: log-weights off by d_i change log N_eff by at
    most 2 (max d - min d), so the bound is exp(2 spread(d)) - 1 over the
    particles that carry weight, plus 1e-6 for the float sums.
  * resampling: bit-exact ancestors and group offsets when both sides resample
    from the same float32 log-weights.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as orc

MEAN_RTOL = 1e-4
LOGEV_RTOL = 1e-5


def f32(v):
    return float(np.float32(v))


def paired_models(ppf, **kw):
    base = dict(width=128, height=128, patch_radius=4, psf_sigma=1.5, amplitude=50.0, background=10.0,
                sigma_xi=math.sqrt(10.0), sigma_m=0.5, sigma_v=0.1, sigma_I=1.0, v0_max=1.0, seed=0,
                filter_id=0)
    base.update(kw)
    fl = {k: (f32(v) if isinstance(v, float) else v) for k, v in base.items()}
    fd = dict(fl)
    gm = ppf.Model(**fd)
    om = orc.Model(**{k: v for k, v in fl.items() if k != "frame_dtype"})
    return gm, om


def check_propagation(om, k, P, anc, S, sigmas):
    """P: (6, N) parents as float64, S: (6, N) GPU propagated state."""
    ref = orc.propagate(om, k, P, anc, np.zeros(P.shape[1]))
    par = P[:, anc]
    scale = np.abs(par[:5]).copy()
    scale[0] += np.abs(par[2])
    scale[1] += np.abs(par[3])
    got, want = S[:5], ref[:5]
    # non-finite parents give non-finite children: the same NaNs and the same
    # infinities on both sides, and no NaN may hide in the tolerance test
    assert np.array_equal(np.isnan(got), np.isnan(want)), "propagation: NaN pattern differs"
    inf = np.isinf(want)
    assert np.array_equal(got[inf], want[inf]), "propagation: infinite values differ"
    fin = np.isfinite(want)
    with np.errstate(invalid="ignore", over="ignore"):
        tol = 2e-6 * (scale + 6.0 * np.array(sigmas)[:, None] + 1.0)
        err = np.where(fin, np.abs(np.where(fin, got, 0.0) - np.where(fin, want, 0.0)), 0.0)
    bad = fin & ~(err <= tol)
    assert not bad.any(), f"propagation: {bad.sum()} mismatches, max err {err.max():.3e}"
    return ref


def loglik_tol(l_ref, I0, r, sxi):
    P = (2 * r + 1) ** 2
    return 1e-5 * np.maximum(1.0, np.abs(l_ref)) + 1e-6 * I0 * I0 * P / (sxi * sxi)


def check_estimate(est, so, W, H, A, d_spread=0.0, d_range=(0.0, 0.0)):
    """so: the oracle's summary of the oracle's log-weights lw_i; the GPU's are
    lw_i + d_i, with d_i in d_range over the particles within 40 of the
    maximum (the rest weigh below e^-40).  log sum exp(lw_i + d_i) - log sum
    exp(lw_i) lies in [min d, max d], so the log-evidence may move by that
    much on top of the summary's own rounding."""
    scale = np.array([W, H, 1.0, 1.0, A])
    ref = np.asarray(so["mean"])
    got = np.asarray(est.mean)
    tol = MEAN_RTOL * np.maximum(np.abs(ref), scale)
    assert np.all(np.abs(got - ref) <= tol), (got, ref)
    le = so["log_evidence"]
    lt = LOGEV_RTOL * max(abs(le), 1.0)
    assert le + d_range[0] - lt <= est.log_evidence <= le + d_range[1] + lt, (est.log_evidence, le, d_range)
    ess_tol = math.expm1(2.0 * d_spread) + 1e-6
    assert abs(est.ess - so["ess"]) <= ess_tol * so["ess"], (est.ess, so["ess"], ess_tol)


def lockstep(pf, gm, om, frames_np, frames_gpu, scheme, K, alpha=0.1, check_resample=True, log=None,
             ess_threshold=None):
    """Run K frames on the GPU and check every stage against the oracle.
    With ess_threshold, resampling follows the N_eff test of Alg. 1: the
    GPU's decision must match the oracle's wherever N_eff is not within
    1e-3 of the threshold, and the kept or resampled particles must match
    the oracle's for the decision the GPU took."""
    N = pf.n
    r = gm.patch_radius
    for k in range(1, K + 1):
        st0, anc0, lwp0 = pf.get_particles(state=True, anc=True, lw_prev=True)
        goff0 = pf.groups()
        P = st0.cpu().double().numpy()
        anc = anc0.cpu().numpy()
        lp = lwp0.cpu().double().numpy()
        pf.step(frames_gpu[k - 1], k)
        st1, _, _ = pf.get_particles()
        S = st1.cpu().double().numpy()
        est = pf.estimate()
        # S1: propagation on identical parents and random streams
        check_propagation(om, k, P, anc, S, [gm.sigma_m, gm.sigma_m, gm.sigma_v, gm.sigma_v, gm.sigma_I])
        # S3: likelihood on the GPU's propagated state
        fr = frames_np[k - 1].astype(np.float64)
        l_ref = orc.loglik_many(om, fr, S[0], S[1], S[4])
        lw_ref = lp + l_ref
        tol = loglik_tol(l_ref, S[4], r, gm.sigma_xi) + 4 * np.spacing(np.abs(lw_ref).astype(np.float32))
        with np.errstate(invalid="ignore"):  # -inf against -inf where both sides agree
            err = np.abs(S[5] - lw_ref)
        fin = np.isfinite(lw_ref)
        assert np.array_equal(np.isfinite(S[5]), fin)
        assert np.all(err[fin] <= tol[fin]), f"frame {k}: loglik max err {err[fin].max():.3e}"
        # S4/S5: normalisation, estimate, log-evidence
        so_state = S.copy()
        so_state[5] = lw_ref
        so = orc.summary(so_state, lp)
        wmax = np.max(lw_ref[fin]) if fin.any() else 0.0
        heavy = fin & (lw_ref > wmax - 40.0)
        d = S[5][heavy] - lw_ref[heavy]
        spread = float(d.max() - d.min()) if d.size else 0.0
        d_range = (float(d.min()), float(d.max())) if d.size else (0.0, 0.0)
        check_estimate(est, so, gm.width, gm.height, gm.amplitude, spread, d_range)
        if log is not None:
            log.append((k, est.mean, est.log_evidence, est.ess))
        sch = scheme[k - 1] if isinstance(scheme, (list, tuple)) else scheme  # one scheme, or one per frame
        if sch is None:
            continue
        # S6-S8: resampling from the same float32 log-weights
        ring0 = pf.ring() if sch == orc.ARNA else None
        pf.resample(sch, alpha, ess_threshold)
        _, anc1, lwp1 = pf.get_particles(state=False, anc=True, lw_prev=True)
        goff1 = pf.groups()
        est2 = pf.estimate()
        if not check_resample:
            continue
        lwf = st1[5].cpu().numpy().astype(np.float32)
        kept = bool(est2.status_flags & 16)
        if ess_threshold is not None:
            if abs(so["ess"] - ess_threshold) > 1e-3 * ess_threshold:
                assert kept == (so["ess"] >= ess_threshold), (k, so["ess"], ess_threshold, kept)
            if log is not None:
                log.append(("kept", k, kept))
        else:
            assert not kept
        if kept:  # Alg. 1 without resampling: identity ancestry, weights carried, layout kept
            assert np.array_equal(anc1.cpu().numpy(), np.arange(N, dtype=np.int32))
            assert np.array_equal(lwp1.cpu().numpy(), lwf)
            assert np.array_equal(goff1, goff0)
            assert (est2.links, est2.moved) == (0, 0)
            if ring0 is not None:
                assert np.array_equal(pf.ring(), ring0)  # ARNA keeps its ring on a kept step
            continue
        if sch == orc.ARNA:
            # the object counts as lost when the log-evidence is negative;
            # away from zero both sides must agree, and the oracle follows the
            # decision the GPU took
            lost = bool(est2.status_flags & 32)
            le = so["log_evidence"]
            if abs(le) > 1e-6 * max(1.0, abs(le)):
                assert lost == (le < 0.0), (k, le, lost)
            if log is not None:
                log.append(("lost", k, lost))
            rc, anc_ref, lwr_ref, goff_ref, stats, ring_ref = orc.resample_arna(
                om, N, k, goff0, lwf, lost, ring0, lw_sum=lwf.astype(np.float64), alpha=f32(alpha))
            assert np.array_equal(pf.ring(), ring_ref), f"frame {k}: ring differs"
        else:
            rc, anc_ref, lwr_ref, goff_ref, stats = orc.resample(om, sch, N, k, goff0, lwf,
                                                                 lwf.astype(np.float64), alpha)
        assert rc == 0
        a1 = anc1.cpu().numpy()
        assert np.array_equal(a1, anc_ref), f"frame {k}: {np.sum(a1 != anc_ref)} ancestors differ"
        if log is not None:  # the most offspring any group's particles had
            per_group = np.bincount(np.searchsorted(goff0, a1, side="right") - 1, minlength=len(goff0) - 1)
            log.append(("offspring", k, int(per_group.max())))
            log.append(("tile offspring", k, int(np.bincount(a1 // 4096).max())))
        assert np.array_equal(goff1, goff_ref)
        l1 = lwp1.cpu().double().numpy()
        tol = 1e-5 * np.maximum(1.0, np.abs(lwr_ref))
        assert np.all(np.abs(l1 - lwr_ref) <= tol)
        assert (est2.links, est2.moved) == (int(stats[0]), int(stats[1]))
        assert (est2.max_group, est2.min_group) == (int(stats[2]), int(stats[3]))
