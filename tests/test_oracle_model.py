"""Pins for the oracle's model steps: the eq. 3/eq. 4 patch likelihood against
closed forms and pixel counting, the NCV propagation against its moments, the
prior draw, and the normalisation/estimate/log-evidence against scipy."""
import math

import numpy as np
import pytest

import synth


def model(orc, **kw):
    base = dict(width=32, height=24, patch_radius=4, psf_sigma=1.5, amplitude=50.0,
                background=10.0, sigma_xi=float(np.sqrt(10.0)))
    base.update(kw)
    return orc.Model(**base)


def sep_sumsq(x, cx, r, sigma, lo=0, hi=10**9):
    """sum over the patch columns of g(i)^2 (1-D), columns restricted to [lo, hi)"""
    i = np.arange(cx - r, cx + r + 1)
    i = i[(i >= lo) & (i < hi)]
    return float(np.sum(np.exp(-((i - x) ** 2) / (sigma * sigma))))


@pytest.mark.parametrize("x,y", [(12.0, 11.0), (12.3, 10.8), (15.49, 9.51)])
def test_flat_background_closed_form(orc, x, y):
    m = model(orc)
    Z = np.full((m.height, m.width), m.background)
    I0 = 37.0
    cx, cy = math.floor(x + 0.5), math.floor(y + 0.5)
    # l = -I0^2 sum_S g^2 / (2 sxi^2), with the 2-D sum of g^2 separable
    want = -I0 * I0 * sep_sumsq(x, cx, 4, 1.5) * sep_sumsq(y, cy, 4, 1.5) / (2 * m.sigma_xi ** 2)
    assert orc.loglik(m, Z, x, y, I0) == pytest.approx(want, rel=1e-12)


def test_noise_free_spot_closed_form_and_maximum(orc):
    m = model(orc)
    mv = synth.make_movie(W=m.width, H=m.height, K=1, sigma=1.5, amplitude=40.0,
                          background=10.0, seed=3, noise=False, start_frac=(0.4, 0.6))
    x, y = mv.truth[0, 0], mv.truth[0, 1]
    Z = mv.frames[0].astype(np.float64)
    cx, cy = math.floor(x + 0.5), math.floor(y + 0.5)
    # noise-free data at the truth: l = +sum_S a^2 / (2 sxi^2), a = I0 g
    want = 40.0 ** 2 * sep_sumsq(x, cx, 4, 1.5) * sep_sumsq(y, cy, 4, 1.5) / (2 * m.sigma_xi ** 2)
    # the generator stores float32 photon counts: allow for that rounding
    assert orc.loglik(m, Z, x, y, 40.0) == pytest.approx(want, rel=2e-6)
    best = orc.loglik(m, Z, x, y, 40.0)
    for dx, dy, dI in [(0.05, 0, 0), (0, -0.05, 0), (0, 0, 1.0), (0, 0, -1.0), (0.03, 0.03, 0)]:
        if math.floor(x + dx + 0.5) == cx and math.floor(y + dy + 0.5) == cy:
            assert orc.loglik(m, Z, x + dx, y + dy, 40.0 + dI) < best


def count_pixels(orc, m, x, y):
    """With a very wide PSF (g == 1 to 1e-12), I0 = 1 and Z = bg, every in-image
    patch pixel contributes exactly 1 to the residual difference."""
    wide = model(orc, width=m.width, height=m.height, patch_radius=m.patch_radius, psf_sigma=1e7)
    Z = np.full((m.height, m.width), m.background)
    return -orc.loglik(wide, Z, x, y, 1.0) * 2 * wide.sigma_xi ** 2


@pytest.mark.parametrize("r", [0, 1, 4, 5])
def test_patch_shape_and_image_border(orc, r):
    m = model(orc, patch_radius=r)
    P = (2 * r + 1)
    assert count_pixels(orc, m, 12.0, 11.0) == pytest.approx(P * P, abs=1e-6)
    assert count_pixels(orc, m, 0.0, 0.0) == pytest.approx((r + 1) ** 2, abs=1e-6)
    assert count_pixels(orc, m, m.width - 1.0, 5.0 + r) == pytest.approx((r + 1) * P, abs=1e-6)
    # anchor c = floor(x + 1/2): -0.5 belongs to column 0, below it to column -1
    assert count_pixels(orc, m, -0.5, 12.0) == pytest.approx((r + 1) * P, abs=1e-6)
    assert count_pixels(orc, m, -0.5000001, 12.0) == pytest.approx(r * P, abs=1e-6)
    # fully outside: empty sum
    assert count_pixels(orc, m, -r - 1.0, 12.0) == 0.0
    assert orc.loglik(m, np.zeros((m.height, m.width)), 1e6, 3.0, 5.0) == 0.0


def test_single_hot_pixel_membership(orc):
    m = model(orc, psf_sigma=1e7)
    r = m.patch_radius
    h = 3.0
    for (px, py) in [(12 + r, 11), (12 - r, 11 - r), (12 + r + 1, 11), (12, 11 + r + 1)]:
        Z = np.full((m.height, m.width), m.background)
        Z[py, px] += h
        inside = abs(px - 12) <= r and abs(py - 11) <= r
        # sum_S [(Zb - 1)^2 - Zb^2] = count - 2 h [p in S]
        want = -((2 * r + 1) ** 2 - (2 * h if inside else 0.0)) / (2 * m.sigma_xi ** 2)
        assert orc.loglik(m, Z, 12.0, 11.0, 1.0) == pytest.approx(want, rel=1e-9)


def test_non_finite_state_has_zero_weight(orc):
    m = model(orc)
    Z = np.zeros((m.height, m.width))
    assert orc.loglik(m, Z, float("nan"), 3.0, 1.0) == -math.inf
    assert orc.loglik(m, Z, 3.0, float("inf"), 1.0) == -math.inf
    assert orc.loglik(m, Z, 3.0, 3.0, float("nan")) == -math.inf


def test_init_prior_ranges(orc):
    stats = pytest.importorskip("scipy.stats")
    m = model(orc, v0_max=0.75, amplitude=20.0)
    st = orc.init(m, 20000)
    x, y, vx, vy, I0, lw = st
    assert stats.kstest((x + 0.5) / m.width, "uniform").pvalue > 1e-4
    assert stats.kstest((y + 0.5) / m.height, "uniform").pvalue > 1e-4
    assert stats.kstest((vx + 0.75) / 1.5, "uniform").pvalue > 1e-4
    assert stats.kstest((I0 - 10.0) / 20.0, "uniform").pvalue > 1e-4
    assert np.all(lw == 0.0)
    assert abs(np.corrcoef(x, y)[0, 1]) < 0.03


def test_propagation_moments(orc):
    m = model(orc, sigma_m=0.5, sigma_v=0.2, sigma_I=1.5)
    N = 60000
    parent = np.zeros((6, N))
    parent[:, 0] = [5.0, 7.0, 0.75, -0.25, 30.0, -2.0]
    anc = np.zeros(N, dtype=np.int32)
    lw_prev = np.full(N, -1.25)
    st = orc.propagate(m, 4, parent, anc, lw_prev)
    want_mean = [5.75, 6.75, 0.75, -0.25, 30.0]
    want_sd = [0.5, 0.5, 0.2, 0.2, 1.5]
    for c in range(5):
        se = want_sd[c] / math.sqrt(N)
        assert abs(st[c].mean() - want_mean[c]) < 5 * se
        assert abs(st[c].std() / want_sd[c] - 1.0) < 0.02
    C = np.corrcoef(st[:5])
    assert np.max(np.abs(C - np.eye(5))) < 0.03
    assert np.all(st[5] == -1.25)


def test_propagation_follows_ancestors(orc):
    m = model(orc, sigma_m=0.0, sigma_v=0.0, sigma_I=0.0)
    rng = np.random.default_rng(0)
    N = 50
    parent = rng.normal(size=(6, N))
    anc = rng.integers(0, N, size=N).astype(np.int32)
    st = orc.propagate(m, 1, parent, anc, np.zeros(N))
    assert np.allclose(st[0], parent[0, anc] + parent[2, anc], rtol=0, atol=1e-15)
    assert np.allclose(st[1], parent[1, anc] + parent[3, anc], rtol=0, atol=1e-15)
    assert np.array_equal(st[2:5], parent[2:5, anc])


def test_summary_against_scipy(orc):
    special = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(5)
    N = 3000
    st = rng.normal(size=(6, N)) * [[3], [2], [1], [1], [5], [4]]
    lw_prev = rng.normal(size=N) - 7.0
    s = orc.summary(st, lw_prev)
    w = special.softmax(st[5])
    assert s["mean"] == pytest.approx(st[:5] @ w, rel=1e-12, abs=1e-12)
    assert s["ess"] == pytest.approx(1.0 / np.sum(w * w), rel=1e-12)
    want = special.logsumexp(st[5]) - special.logsumexp(lw_prev)
    assert s["log_evidence"] == pytest.approx(want, rel=1e-12)
    assert s["max_lw"] == st[5].max()


def test_summary_special_cases(orc):
    N = 64
    st = np.zeros((6, N))
    st[0] = np.arange(N)
    st[5] = -3.5
    s = orc.summary(st, np.zeros(N))
    assert s["ess"] == pytest.approx(N, rel=1e-14)
    assert s["log_evidence"] == pytest.approx(-3.5, abs=1e-13)
    assert s["mean"][0] == pytest.approx((N - 1) / 2, rel=1e-14)
    st[5] = -np.inf
    st[5, 17] = 2.0
    s = orc.summary(st, np.zeros(N))
    assert s["ess"] == 1.0 and s["mean"][0] == 17.0
    assert s["log_evidence"] == pytest.approx(2.0 - math.log(N), abs=1e-13)


def test_sampled_propagation_and_likelihood_match_full(orc):
    """The per-slot helpers used at full size equal the whole-array routines."""
    m = model(orc, sigma_m=0.4, sigma_v=0.1, sigma_I=0.7)
    rng = np.random.default_rng(9)
    N = 300
    parent = rng.normal(size=(6, N)) * [[4], [4], [1], [1], [5], [1]] + [[15], [11], [0], [0], [30], [0]]
    anc = rng.integers(0, N, size=N).astype(np.int32)
    full = orc.propagate(m, 6, parent, anc, np.zeros(N))
    slots = np.array([0, 7, 299, 123])
    got = orc.propagate_slots(m, 6, slots, parent[:5, anc[slots]])
    assert np.array_equal(got, full[:5, slots])
    Z = rng.poisson(12.0, size=(m.height, m.width)).astype(np.float64)
    l = orc.loglik_many(m, Z, full[0], full[1], full[4])
    w = orc.weight(m, Z, full)
    assert np.array_equal(l, w[5] - full[5])


def test_summary_ignores_zero_weight_particles(orc):
    """Zero-weight particles (lw = -inf or NaN) are outside the weighted-sample
    approximation: their state, even non-finite, does not enter the estimate."""
    N = 6
    st = np.zeros((6, N))
    st[0] = [1.0, 3.0, np.inf, np.nan, 1e300, 5.0]
    st[5] = [0.0, 0.0, -np.inf, np.nan, -1e6, -np.inf]
    s = orc.summary(st, np.zeros(N))
    assert s["mean"][0] == pytest.approx(2.0, abs=1e-12)
    assert s["ess"] == pytest.approx(2.0, rel=1e-12)
    assert s["log_evidence"] == pytest.approx(math.log(2.0) - math.log(6.0), abs=1e-12)


# ------------------------------------------------------------------ pcSIR
def test_piecewise_constant_likelihood_cells(orc):
    """pcSIR: the likelihood is constant on every pixel cell [c - 1/2, c + 1/2)^2
    and equals the eq. 4 likelihood at the cell centre; the flat-frame closed
    form holds at the centre for every point of the cell."""
    m_ex = model(orc)
    m_pc = model(orc, likelihood=1)
    rng = np.random.default_rng(5)
    Z = rng.poisson(15.0, size=(m_ex.height, m_ex.width)).astype(np.float64)
    for cx, cy in [(12, 11), (0, 0), (31, 23), (-3, 5), (34, 25)]:
        I0 = float(rng.uniform(10, 60))
        centre = orc.loglik(m_ex, Z, float(cx), float(cy), I0)
        for _ in range(6):
            x = cx + float(rng.uniform(-0.5, 0.5))
            y = cy + float(rng.uniform(-0.5, 0.5))
            assert orc.loglik(m_pc, Z, x, y, I0) == centre
    flat = np.full((m_pc.height, m_pc.width), m_pc.background)
    want = -30.0 ** 2 * sep_sumsq(12, 12, 4, 1.5) * sep_sumsq(11, 11, 4, 1.5) / (2 * m_pc.sigma_xi ** 2)
    assert orc.loglik(m_pc, flat, 12.37, 10.62, 30.0) == pytest.approx(want, rel=1e-12)
    assert orc.loglik(m_pc, flat, math.nan, 1.0, 30.0) == -math.inf


def test_piecewise_constant_filter_tracks(orc):
    """End to end: the oracle's SIR with the pcSIR likelihood follows the spot
    to within the cell quantisation (parity with the cited pcSIR paper is not
    pinned; this is a sanity check of the reading)."""
    mv = synth.make_movie(W=64, H=64, K=12, sigma=1.5, amplitude=50.0, background=10.0, seed=2)
    m = orc.Model(width=64, height=64, patch_radius=4, psf_sigma=1.5, amplitude=50.0, background=10.0,
                  sigma_xi=math.sqrt(200.0), sigma_m=0.5, sigma_v=0.1, sigma_I=1.0, seed=4, likelihood=1)
    rc, est, _ = orc.run(m, 8192, mv.frames)
    assert rc == 0
    err = est[4:, :2] - mv.truth[4:, :2]
    assert np.sqrt((err ** 2).sum(1).mean()) < 0.8
