"""Pins for the oracle's resampling (Alg. 1 resampling step, Sec. 3-4):
fixed-point weights against 2^x, systematic tickets against brute-force
enumeration, the schedulers of Alg. 2-4 on hand-worked cases and invariants,
RPA's independence of the group count and RNA's structure."""
import math

import numpy as np
import pytest


def test_exp2_fraction_accuracy(orc):
    f = np.linspace(0.0, 1.0, 4097, dtype=np.float32)[:-1]
    p = np.array([orc.exp2_frac(v) for v in f])
    rel = np.abs(p / np.exp2(f.astype(np.float64)) - 1.0)
    assert rel.max() < 3e-7
    assert orc.exp2_frac(0.0) == 1.0


def test_quantiser_properties(orc):
    s = orc.scale_bits(1000)
    assert s == 63 - 10
    assert orc.scale_bits(1) == 63 and orc.scale_bits(2) == 62 and orc.scale_bits(1024) == 53
    lw = np.sort(np.random.default_rng(1).normal(scale=8.0, size=2000)).astype(np.float32)
    M = float(lw.max())
    q = orc.quantise(lw, M, s)
    assert int(q[-1]) == 2**s                       # the maximum maps to 2^s
    assert np.all(np.diff(q.astype(np.float64)) >= 0)  # monotone in the weight
    exact = np.exp2(s) * np.exp(lw.astype(np.float64) - M)
    big = exact > 2**20
    # float32 rounding of d = lw - M and of t = d log2(e) moves t by up to
    # ~2 |t| 2^-24, i.e. a relative error of ln2 * 2|t| 2^-24 in 2^t, plus
    # the polynomial's 3e-7
    t = np.abs((lw.astype(np.float64) - M) / math.log(2.0))
    bound = 3e-7 + math.log(2.0) * 2.0 * (t + 1.0) * 2.0**-24
    assert np.all(np.abs(q[big] / exact[big] - 1.0) < bound[big])
    assert np.all(q <= np.floor(exact * (1 + bound)) + 1)
    assert orc.quantise([np.nan], 0.0, s)[0] == 0
    assert orc.quantise([-np.inf], 0.0, s)[0] == 0
    assert orc.quantise([-200.0], 0.0, s)[0] == 0


def test_balanced_offsets_reading_r14(orc):
    """R14's targets n_g = floor(N/G) + [g < N mod G]: hand cases, then sizes
    that differ by at most one with the larger groups first, for every G <= N."""
    assert list(orc.balanced_offsets(10, 4)) == [0, 3, 6, 8, 10]
    assert list(orc.balanced_offsets(7, 7)) == list(range(8))
    assert list(orc.balanced_offsets(9, 1)) == [0, 9]
    for N in range(1, 60):
        for G in range(1, N + 1):
            off = orc.balanced_offsets(N, G)
            sz = np.diff(off)
            assert off[0] == 0 and off[-1] == N
            assert sz.max() - sz.min() <= 1 and sz.min() == N // G
            assert np.all(np.diff(sz) <= 0)  # the N mod G larger groups come first


def test_tickets_below_brute_force(orc):
    rng = np.random.default_rng(2)
    for _ in range(300):
        n = int(rng.integers(1, 40))
        Q = int(rng.integers(1, 10**6))
        u = int(rng.integers(0, Q))
        c = int(rng.integers(0, Q + 1))
        want = sum(1 for j in range(n) if u + j * Q < n * c)
        assert orc.tickets_below(c, n, u, Q) == want


def test_systematic_enumeration_n8(orc):
    """Every offset u in [0, Q): ticket counts equal direct counting, and summed
    over u each particle gets exactly N q_i tickets (unbiasedness, in integers)."""
    rng = np.random.default_rng(3)
    N = 8
    for trial in range(4):
        q = rng.integers(0, 300, size=N).astype(np.uint64)
        q[rng.integers(0, N)] = 0
        Q = int(q.sum())
        C = np.cumsum(q.astype(np.int64))
        total = np.zeros(N, dtype=np.int64)
        for u in range(Q):
            rc, anc, off = orc.systematic(q, u)
            assert rc == 0
            direct = np.zeros(N, dtype=np.int64)
            for j in range(N):
                pos = u + j * Q
                i = next(i for i in range(N) if N * int(C[i]) > pos)
                direct[i] += 1
                assert anc[j] == i
            assert np.array_equal(off, direct)
            total += off
        assert np.array_equal(total, N * q.astype(np.int64))


def test_systematic_invariants(orc):
    rng = np.random.default_rng(4)
    for N in [1, 7, 1000, 4096]:
        q = (rng.random(N) ** 4 * 2**40).astype(np.uint64)
        q[rng.random(N) < 0.2] = 0
        if q.sum() == 0:
            q[0] = 1
        Q = int(q.sum())
        u = int(rng.integers(0, Q))
        rc, anc, off = orc.systematic(q, u)
        assert rc == 0 and off.sum() == N
        share = N * q.astype(object) / Q
        for i in range(N):
            assert math.floor(share[i]) <= off[i] <= math.ceil(share[i])
        assert np.all(np.diff(anc) >= 0)
        assert np.all(q[anc] > 0)


def test_systematic_degenerate(orc):
    rc, anc, off = orc.systematic(np.zeros(5, dtype=np.uint64), 0)
    assert rc == orc.EDEGENERATE


def _offset_words(orc, cases):
    """Philox words of the ticket-offset counters: triton's when its CPU
    interpreter runs, else the oracle's own (pinned against triton by
    test_philox_matches_triton_reference)."""
    from philox_ref import triton_philox
    ref, _ = triton_philox(cases)
    if ref is not None:
        return ref
    return [[orc.philox(c, [seed & 0xFFFFFFFF, seed >> 32]).tolist() for c in ctrs] for seed, ctrs in cases]


def test_ticket_offset_is_high_word_of_r64_times_q(orc):
    """R2: u = floor(r64 Q / 2^64) with r64 = w1 2^32 + w0, (w0, w1) the
    first two words of Philox4x32-10 with key (seed_lo, seed_hi) and counter
    (index, frame, filter, purpose << 8).  The product is formed here with
    Python integers from independently computed Philox words, so swapped
    words, a 32-bit r64 or the low half of the product all fail."""
    rng = np.random.default_rng(77)
    seeds = [9, 2**40 + 3, 0xDEADBEEFCAFEF00D]
    cases = []
    for seed in seeds:
        ctrs = []
        for j in range(8):
            purpose = orc.PURPOSE_RESAMPLE if j % 2 == 0 else orc.PURPOSE_GROUP_RESAMPLE
            index = 0 if purpose == orc.PURPOSE_RESAMPLE else int(rng.integers(0, 20000))
            frame = int(rng.integers(1, 2**31))
            filt = int(rng.integers(0, 5000)) if j >= 4 else 0
            ctrs.append([index, frame, filt, purpose << 8])
        cases.append([seed, ctrs])
    words = _offset_words(orc, cases)
    Qs = [1, 3, 2**40 + 7, 2**63, 2**64 - 1, int(rng.integers(1, 2**62))]
    for (seed, ctrs), ws in zip(cases, words):
        for (index, frame, filt, pw), w in zip(ctrs, ws):
            r64 = (int(w[1]) << 32) | int(w[0])
            for Q in Qs:
                want = (r64 * Q) >> 64
                got = orc.ticket_offset(seed, filt, frame, pw >> 8, index, Q)
                assert got == want, (seed, index, frame, filt, pw >> 8, Q, got, want)
                assert 0 <= got < Q


def test_ticket_offset_is_uniform(orc):
    """u / Q over 10^4 frames is uniform on [0, 1) (Kolmogorov-Smirnov at
    large Q), and u is uniform on {0, 1, 2} at Q = 3 (chi-square)."""
    stats = pytest.importorskip("scipy.stats")
    K = 10_000
    for Q in [2**63, 2**40 + 7]:
        u = np.array([orc.ticket_offset(5, 0, k, orc.PURPOSE_RESAMPLE, 0, Q) for k in range(1, K + 1)],
                     dtype=np.float64) / float(Q)
        assert stats.kstest(u, "uniform").pvalue > 1e-4
    g = np.array([orc.ticket_offset(5, 3, 17, orc.PURPOSE_GROUP_RESAMPLE, i, 2**50) for i in range(K)],
                 dtype=np.float64) / 2.0**50
    assert stats.kstest(g, "uniform").pvalue > 1e-4
    c = np.bincount([orc.ticket_offset(11, 0, k, orc.PURPOSE_RESAMPLE, 0, 3) for k in range(1, K + 1)],
                    minlength=3)
    assert c.sum() == K and len(c) == 3
    assert stats.chisquare(c).pvalue > 1e-4


# ---------------------------------------------------------------- schedulers
COUNT = np.array([9, 0, 3, 6, 2])
TARGET = np.array([4, 4, 4, 4, 4])


def links(orc, scheme, count=COUNT, target=TARGET):
    s, d, c = orc.schedule(scheme, count, target)
    return list(zip(s.tolist(), d.tolist(), c.tolist()))


def test_greedy_hand_case(orc):
    # senders g0 (+5), g3 (+2); receivers g1 (-4), g2 (-1), g4 (-2), in group order
    assert links(orc, orc.RPA_GS) == [(0, 1, 4), (0, 2, 1), (3, 4, 2)]


def test_sorted_greedy_hand_case(orc):
    # receivers sorted by deficit: g1 (4), g4 (2), g2 (1)
    assert links(orc, orc.RPA_SGS) == [(0, 1, 4), (0, 4, 1), (3, 4, 1), (3, 2, 1)]


def test_largest_gradient_hand_case(orc):
    # rank pairs (g0, g1) and (g3, g4); C = min(|S|, |R|) = 2 links
    assert links(orc, orc.RPA_LGS) == [(0, 1, 4), (3, 4, 2)]


def apply(count, target, L):
    out = count.astype(np.int64).copy()
    for s, d, c in L:
        out[s] -= c
        out[d] += c
    return out


@pytest.mark.parametrize("seed", range(6))
def test_scheduler_invariants(orc, seed):
    rng = np.random.default_rng(seed)
    G = int(rng.integers(2, 60))
    target = rng.integers(5, 50, size=G)
    N = int(target.sum())
    count = np.bincount(rng.choice(G, size=N, p=rng.dirichlet(np.ones(G) * 0.3)), minlength=G)
    nS = int((count > target).sum())
    nR = int((count < target).sum())
    for scheme in (orc.RPA_GS, orc.RPA_SGS):
        L = links(orc, scheme, count, target)
        assert all(c > 0 and count[s] > target[s] and count[d] < target[d] for s, d, c in L)
        assert np.array_equal(apply(count, target, L), target)       # perfect balance
        assert len(L) <= nS + nR - 1 or (nS + nR == 0 and not L)
    L = links(orc, orc.RPA_LGS, count, target)
    assert len(L) == min(nS, nR)                                      # C = min(|S|,|R|)
    after = apply(count, target, L)
    assert after.sum() == N
    sur = np.maximum(count - target, 0)
    dfc = np.maximum(target - count, 0)
    for s, d, c in L:
        assert c == min(sur[s], dfc[d])


# ---------------------------------------------------------------- RPA / RNA
def weights(N, seed, spread=6.0):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=N) * spread).astype(np.float32)


@pytest.mark.parametrize("scheme", ["RPA_GS", "RPA_SGS", "RPA_LGS"])
def test_rpa_ancestors_do_not_depend_on_group_count(orc, scheme):
    m = orc.Model(seed=11)
    N = 3000
    lw = weights(N, 1)
    rc, sys_anc, _, _, _ = orc.resample(m, orc.SYSTEMATIC, N, 5, orc.balanced_offsets(N, 1), lw)
    assert rc == 0
    for G in [1, 7, 64]:
        goff = orc.balanced_offsets(N, G)
        rc, anc, lwr, gout, st = orc.resample(m, getattr(orc, scheme), N, 5, goff, lw)
        assert rc == 0
        assert np.array_equal(np.sort(anc), sys_anc)
        assert np.all(lwr == 0.0)
        assert gout[0] == 0 and gout[-1] == N and np.all(np.diff(gout) >= 0)
        if scheme != "RPA_LGS":
            assert np.array_equal(gout, goff)
        # every group's first slots are its own offspring
        for g in range(G):
            own = anc[gout[g]:gout[g + 1]]
            mine = (own >= goff[g]) & (own < goff[g + 1])
            k = int(mine.sum())
            assert np.all(mine[:k])


def test_rpa_lgs_imbalance_and_link_count(orc):
    m = orc.Model(seed=2)
    N, G = 4000, 40
    lw = weights(N, 3, spread=3.0)
    lw[:500] += 6.0          # the first groups are much heavier
    goff = orc.balanced_offsets(N, G)
    rc, anc, _, gout, st = orc.resample(m, orc.RPA_LGS, N, 1, goff, lw)
    sizes = np.diff(gout)
    assert rc == 0 and sizes.sum() == N and sizes.max() > 100
    rc2, anc2, _, gout2, st2 = orc.resample(m, orc.RPA_GS, N, 1, goff, lw)
    assert np.array_equal(np.diff(gout2), np.full(G, 100))
    assert st[0] <= st2[0]        # LGS never needs more links than GS


def test_rna_structure(orc):
    m = orc.Model(seed=4)
    N, G = 1000, 8
    goff = orc.balanced_offsets(N, G)
    lw = weights(N, 6, spread=2.0)
    rc, anc, lwr, gout, st = orc.resample(m, orc.RNA, N, 2, goff, lw, alpha=0.1)
    assert rc == 0 and np.array_equal(gout, goff)
    mig = int(math.floor(0.1 * 125))
    for g in range(G):
        lo, hi = goff[g], goff[g + 1]
        p = (g - 1) % G
        assert np.all((anc[lo:hi - mig] >= lo) & (anc[lo:hi - mig] < hi))
        assert np.all((anc[hi - mig:hi] >= goff[p]) & (anc[hi - mig:hi] < goff[p + 1]))
    # total post-resampling weight is 1
    assert np.log(np.exp(lwr).sum()) == pytest.approx(0.0, abs=1e-12)
    # each group's weight is carried by its own offspring
    special = pytest.importorskip("scipy.special")
    lws = lw.astype(np.float64)
    for g in range(G):
        want = special.logsumexp(lws[goff[g]:goff[g + 1]]) - special.logsumexp(lws) - math.log(125)
        assert lwr[goff[g]] == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_rna_single_group_is_local_systematic(orc):
    m = orc.Model(seed=8)
    N = 777
    lw = weights(N, 9)
    rc, anc, lwr, _, _ = orc.resample(m, orc.RNA, N, 3, orc.balanced_offsets(N, 1), lw, alpha=0.5)
    q = orc.quantise(lw)
    u = orc.ticket_offset(8, 0, 3, orc.PURPOSE_GROUP_RESAMPLE, 0, int(q.sum()))
    rc2, want, _ = orc.systematic(q, u)
    assert rc == 0 and rc2 == 0 and np.array_equal(anc, want)
    assert np.allclose(lwr, -math.log(N), rtol=0, atol=1e-12)


def test_global_degenerate_keeps_particles(orc):
    m = orc.Model()
    N = 10
    lw = np.full(N, np.nan, dtype=np.float32)
    rc, anc, lwr, gout, _ = orc.resample(m, orc.SYSTEMATIC, N, 1, orc.balanced_offsets(N, 2), lw)
    assert rc == orc.EDEGENERATE and np.array_equal(anc, np.arange(N))


def test_systematic_enumeration_other_ticket_counts(orc):
    """Systematic draws of n tickets over weights of a different length (the
    second stage of two-stage RPA): for every offset u in [0, Q) the parents
    equal direct ticket counting, and summed over u particle i receives
    exactly n q_i tickets (unbiasedness, in integers)."""
    rng = np.random.default_rng(12)
    for n_in, nt in [(6, 4), (5, 9), (7, 1), (3, 3)]:
        q = rng.integers(0, 150, size=n_in).astype(np.uint64)
        q[rng.integers(0, n_in)] += 1
        Q = int(q.sum())
        C = np.cumsum(q.astype(np.int64))
        total = np.zeros(n_in, dtype=np.int64)
        for u in range(Q):
            rc, anc, off = orc.systematic(q, u, n_tickets=nt)
            assert rc == 0
            for j in range(nt):
                pos = u + j * Q
                assert anc[j] == next(i for i in range(n_in) if nt * int(C[i]) > pos)
            total += off
        assert np.array_equal(total, nt * q.astype(np.int64))


@pytest.mark.parametrize("scheme", ["GS", "SGS", "LGS"])
def test_two_stage_rpa(orc, scheme):
    """Two-stage proportional allocation: stage 1 gives every group the same
    number of offspring as one-stage RPA (so the same layout and routing);
    stage 2 draws them inside the group, each particle getting the floor or
    the ceiling of N_g q_i / Q_g; with one group it is the group's own
    systematic draw."""
    m = orc.Model(seed=5)
    N = 3000
    lw = weights(N, 2)
    q = orc.quantise(lw).astype(np.int64)
    one, two = getattr(orc, "RPA_" + scheme), getattr(orc, "RPA2_" + scheme)
    for G in [1, 7, 64]:
        goff = orc.balanced_offsets(N, G)
        rc1, anc1, _, gout1, st1 = orc.resample(m, one, N, 4, goff, lw)
        rc2, anc2, lwr2, gout2, st2 = orc.resample(m, two, N, 4, goff, lw)
        assert rc1 == 0 and rc2 == 0
        assert np.array_equal(gout1, gout2) and np.array_equal(st1, st2) and np.all(lwr2 == 0.0)
        src1 = np.searchsorted(goff, anc1, side="right") - 1
        src2 = np.searchsorted(goff, anc2, side="right") - 1
        Ng = np.bincount(src1, minlength=G)
        assert np.array_equal(Ng, np.bincount(src2, minlength=G))
        off = np.bincount(anc2, minlength=N)
        for g in range(G):
            lo, hi = goff[g], goff[g + 1]
            Qg = int(q[lo:hi].sum())
            if Ng[g] == 0:
                continue
            exact = Ng[g] * q[lo:hi] / Qg
            assert np.all(off[lo:hi] >= np.floor(exact) - 1e-9) and np.all(off[lo:hi] <= np.ceil(exact) + 1e-9)
        if G == 1:
            u = orc.ticket_offset(5, 0, 4, orc.PURPOSE_GROUP_RESAMPLE, 0, int(q.sum()))
            rc, want, _ = orc.systematic(q.astype(np.uint64), u)
            assert np.array_equal(anc2, want)
