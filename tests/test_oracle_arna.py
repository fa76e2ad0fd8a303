"""Pins for the oracle's ARNA (Sec. 7: RNA with an exchange ratio that follows
the number of groups involved in tracking, and a ring order redrawn when the
object is lost).  The paper describes ARNA in words only, so these pin the
reading taken, piece by piece, against independently pinned parts: the
ring against Philox (pinned by known-answer tests), the involved groups
against the global systematic draw (pinned by enumeration), the exchange
against RNA's local draws."""
import math

import numpy as np
import pytest


def weights(N, seed, spread=4.0):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=N) * spread).astype(np.float32)


def expected_exchange(orc, m, N, frame, goff, lw, mig, ring):
    """RNA's local offspring (no exchange), then the last mig of every group
    moved to the tail of its successor on the ring."""
    G = len(goff) - 1
    rc, local, lwl, _, _ = orc.resample(m, orc.RNA, N, frame, goff, lw, alpha=0.0)
    assert rc == 0
    succ = np.empty(G, dtype=np.int64)
    succ[ring] = np.roll(ring, -1)
    anc = np.empty(N, dtype=np.int32)
    lwr = np.empty(N)
    for g in range(G):
        lo, hi = goff[g], goff[g + 1]
        sz = hi - lo
        keep = sz - mig
        anc[lo:lo + keep] = local[lo:lo + keep]
        lwr[lo:lo + keep] = lwl[lo:lo + keep]
        n = succ[g]
        nlo, nhi = goff[n], goff[n + 1]
        anc[nhi - mig:nhi] = local[lo + keep:hi]
        lwr[nhi - mig:nhi] = lwl[lo + keep:hi]
    return anc, lwr


def involved_groups(orc, m, N, frame, goff, lw):
    rc, sys_anc, _, _, _ = orc.resample(m, orc.SYSTEMATIC, N, frame, goff, lw)
    assert rc == 0
    src = np.searchsorted(goff, sys_anc, side="right") - 1
    o = np.bincount(src, minlength=len(goff) - 1)
    return int(np.sum(o >= np.diff(goff)))


def test_ring_is_philox_order(orc):
    seed, fid, frame, G = 77, 3, 9, 40
    ring = orc.arna_ring(seed, fid, frame, G)
    assert np.array_equal(np.sort(ring), np.arange(G))
    key = [(seed & 0xFFFFFFFF), seed >> 32]
    words = [int(orc.philox([g, frame, fid, (orc.PURPOSE_RING << 8) | 0], key)[0]) for g in range(G)]
    want = sorted(range(G), key=lambda g: (words[g], g))
    assert list(ring) == want
    # another frame or filter gives another order
    assert not np.array_equal(ring, orc.arna_ring(seed, fid, frame + 1, G))
    assert not np.array_equal(ring, orc.arna_ring(seed, fid + 1, frame, G))


@pytest.mark.parametrize("G", [1, 5, 16])
def test_not_lost_is_rna_with_adaptive_ratio(orc, G):
    m = orc.Model(seed=21)
    N, frame, alpha = 1600, 4, 0.5
    goff = orc.balanced_offsets(N, G)
    lw = weights(N, G)
    lw[goff[min(2, G - 1)]:goff[min(2, G - 1) + 1]] += 3.0   # one heavier group
    ring = np.arange(G, dtype=np.int32)
    rc, anc, lwr, gout, st, ring_out = orc.resample_arna(m, N, frame, goff, lw, False, ring, alpha=alpha)
    assert rc == 0 and np.array_equal(gout, goff) and np.array_equal(ring_out, ring)
    inv = involved_groups(orc, m, N, frame, goff, lw)
    minsz = int(np.diff(goff).min())
    mig = int(math.floor(alpha * (G - inv) * minsz / G))
    assert st[4] == inv and 1 <= inv <= G
    assert st[1] == (mig * G if G > 1 else 0) and st[0] == (G if (G > 1 and mig > 0) else 0)
    want_anc, want_lwr = expected_exchange(orc, m, N, frame, goff, lw, mig, ring)
    assert np.array_equal(anc, want_anc)
    assert np.array_equal(lwr, want_lwr)
    if G > 1:
        assert mig > 0   # the heavy group leaves others below their share


def test_lost_redraws_the_ring_before_the_exchange(orc):
    m = orc.Model(seed=5, filter_id=2)
    N, G, frame = 1200, 12, 7
    goff = orc.balanced_offsets(N, G)
    lw = weights(N, 3)
    ring_in = np.arange(G, dtype=np.int32)[::-1].copy()
    rc, anc, lwr, _, st, ring_out = orc.resample_arna(m, N, frame, goff, lw, True, ring_in, alpha=0.4)
    assert rc == 0
    ring = orc.arna_ring(5, 2, frame, G)
    assert np.array_equal(ring_out, ring)
    inv = involved_groups(orc, m, N, frame, goff, lw)
    mig = int(math.floor(0.4 * (G - inv) * 100 / G))
    want_anc, want_lwr = expected_exchange(orc, m, N, frame, goff, lw, mig, ring)
    assert np.array_equal(anc, want_anc) and np.array_equal(lwr, want_lwr)


def test_equal_weights_involve_every_group(orc):
    """Equal weights give every particle one ticket: o_g = n_g for every
    group, so the ratio drops to zero and nothing moves."""
    m = orc.Model(seed=1)
    N, G = 1000, 10
    goff = orc.balanced_offsets(N, G)
    lw = np.zeros(N, dtype=np.float32)
    rc, anc, _, _, st, _ = orc.resample_arna(m, N, 2, goff, lw, False, np.arange(G, dtype=np.int32), alpha=0.5)
    assert rc == 0 and st[4] == G and st[1] == 0 and st[0] == 0
    assert np.array_equal(anc, np.arange(N))


def test_one_heavy_particle_involves_one_group(orc):
    m = orc.Model(seed=1)
    N, G = 1000, 10
    goff = orc.balanced_offsets(N, G)
    lw = np.full(N, -200.0, dtype=np.float32)
    lw[437] = 0.0
    rc, anc, _, _, st, _ = orc.resample_arna(m, N, 2, goff, lw, False, np.arange(G, dtype=np.int32), alpha=0.5)
    assert rc == 0 and st[4] == 1
    assert st[1] == math.floor(0.5 * 9 * 100 / 10) * G


def test_unusable_weights_involve_no_group(orc):
    m = orc.Model(seed=1)
    N, G = 100, 4
    goff = orc.balanced_offsets(N, G)
    lw = np.full(N, -np.inf, dtype=np.float32)
    rc, anc, lwr, _, st, _ = orc.resample_arna(m, N, 2, goff, lw, False, np.arange(G, dtype=np.int32), alpha=0.2)
    assert rc == 0 and st[4] == 0 and st[1] == 5 * G
    # every group keeps its own particles (none has usable weight); the
    # exchange still moves the last 5 of each to the next group
    want_anc, _ = expected_exchange(orc, m, N, 2, goff, lw, 5, np.arange(G))
    assert np.array_equal(anc, want_anc)


def test_run_follows_the_ring_state(orc):
    """A whole ARNA run: the oracle's run keeps the ring between frames and
    redraws it on frames whose log-evidence is negative; it finishes and
    tracks like RNA on a movie whose spot never disappears."""
    import synth
    mv = synth.make_movie(W=64, H=64, K=6, seed=3)
    m = orc.Model(width=64, height=64, patch_radius=4, psf_sigma=1.5, amplitude=50.0, background=10.0,
                  sigma_xi=math.sqrt(10.0), sigma_m=0.5, sigma_v=0.1, sigma_I=1.0, seed=3)
    rc, est, _ = orc.run(m, 4096, mv.frames, group_size=512, scheme=orc.ARNA, alpha=0.5)
    assert rc == 0 and np.all(np.isfinite(est))
    err = np.hypot(est[-1, 0] - mv.truth[-1][0], est[-1, 1] - mv.truth[-1][1])
    assert err < 1.0


def test_unequal_groups(orc):
    """An LGS-like layout of unequal groups: the involved test compares each
    group's proportional offspring with its own size, the migrant count uses
    the smallest group, and the exchange follows a permuted ring."""
    m = orc.Model(seed=9)
    N, frame = 2000, 6
    sizes = np.array([500, 120, 380, 260, 740])
    goff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    G = len(sizes)
    lw = weights(N, 5, spread=3.0)
    ring = np.array([3, 0, 4, 1, 2], dtype=np.int32)
    rc, anc, lwr, gout, st, ring_out = orc.resample_arna(m, N, frame, goff, lw, False, ring, alpha=0.5)
    assert rc == 0 and np.array_equal(gout, goff) and np.array_equal(ring_out, ring)
    inv = involved_groups(orc, m, N, frame, goff, lw)
    mig = int(math.floor(0.5 * (G - inv) * 120 / G))
    assert mig > 0, "the case must move particles for the ring to be tested"
    assert st[4] == inv and st[2] == 740 and st[3] == 120 and st[1] == mig * G
    want_anc, want_lwr = expected_exchange(orc, m, N, frame, goff, lw, mig, ring)
    assert np.array_equal(anc, want_anc) and np.array_equal(lwr, want_lwr)
