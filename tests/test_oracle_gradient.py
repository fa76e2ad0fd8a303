"""Pins for the oracle's gradient of the log marginal likelihood estimate
(sum of per-frame log-evidences, systematic resampling held fixed, I0 = A):
per-particle partials against central differences of the likelihood, and the
whole reverse-mode gradient against central differences of the replayed
objective (common random numbers, ancestors and patch anchors replayed)."""
import math

import numpy as np
import pytest

import synth


def model(orc, **kw):
    base = dict(width=48, height=40, patch_radius=4, psf_sigma=1.5, amplitude=30.0, background=10.0,
                sigma_xi=math.sqrt(10.0), sigma_m=0.5, sigma_v=0.1, sigma_I=0.0, seed=3)
    base.update(kw)
    return orc.Model(**base)


def test_partials_match_central_differences(orc):
    m = model(orc)
    rng = np.random.default_rng(0)
    Z = rng.poisson(12.0, size=(m.height, m.width)).astype(np.float64)
    for (x, y, I0) in [(20.3, 17.8, 28.0), (1.2, 2.6, 15.0), (47.4, 0.1, 40.0)]:
        anc = (math.floor(x + 0.5), math.floor(y + 0.5))
        p = orc.loglik_partials(m, Z, x, y, I0, anc)
        assert p[0] == pytest.approx(orc.loglik(m, Z, x, y, I0), rel=1e-13, abs=1e-12)
        h = 1e-6
        def L(**kw):
            mm = model(orc, **{k: v for k, v in kw.items() if k in ("psf_sigma", "background")})
            return orc.loglik_partials(mm, Z, kw.get("x", x), kw.get("y", y), kw.get("I0", I0), anc)[0]
        fd = [
            (L(psf_sigma=1.5 + h) - L(psf_sigma=1.5 - h)) / (2 * h),
            (L(I0=I0 + h) - L(I0=I0 - h)) / (2 * h),
            (L(background=10.0 + h) - L(background=10.0 - h)) / (2 * h),
            (L(x=x + h) - L(x=x - h)) / (2 * h),
            (L(y=y + h) - L(y=y - h)) / (2 * h),
        ]
        for c in range(5):
            assert p[1 + c] == pytest.approx(fd[c], rel=1e-6, abs=1e-6)


def test_background_partial_closed_form(orc):
    """d l / d I_bg = -(I0 / sigma_xi^2) sum_S g for an interior particle:
    the separable closed form of sum_S g."""
    m = model(orc)
    Z = np.full((m.height, m.width), 13.0)
    x, y, I0 = 20.25, 17.5, 22.0
    p = orc.loglik_partials(m, Z, x, y, I0)
    i = np.arange(20 - 4, 20 + 5)
    j = np.arange(18 - 4, 18 + 5)
    sg = np.sum(np.exp(-((i - x) ** 2) / (2 * 1.5 ** 2))) * np.sum(np.exp(-((j - y) ** 2) / (2 * 1.5 ** 2)))
    assert p[3] == pytest.approx(-I0 * sg / m.sigma_xi ** 2, rel=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_replayed_central_differences(orc, seed):
    mv = synth.make_movie(W=48, H=40, K=6, sigma=1.5, amplitude=30.0, background=10.0, seed=seed,
                          start_frac=(0.4, 0.6))
    m = model(orc, seed=seed)
    N = 1500
    theta = np.array([1.5, 30.0, 10.0, 0.5])
    rc, L0, g, anc, anchors = orc.grad_run(m, N, mv.frames, theta)
    assert rc == 0 and np.isfinite(L0)
    rc, L1, g1, _, _ = orc.grad_run(m, N, mv.frames, theta, anc, anchors)
    assert L1 == pytest.approx(L0, rel=1e-14) and np.allclose(g1, g, rtol=1e-13)
    for c, h in enumerate([1e-5, 1e-4, 1e-5, 1e-6]):
        tp, tm = theta.copy(), theta.copy()
        tp[c] += h
        tm[c] -= h
        Lp = orc.grad_run(m, N, mv.frames, tp, anc, anchors)[1]
        Lm = orc.grad_run(m, N, mv.frames, tm, anc, anchors)[1]
        fd = (Lp - Lm) / (2 * h)
        assert g[c] == pytest.approx(fd, rel=1e-5, abs=1e-5 * max(1.0, abs(L0)) * 1e-3), (c, g[c], fd)
