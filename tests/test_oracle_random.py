"""Pins for the oracle's random streams: Philox4x32-10 against an independent
library implementation (triton's, run by its CPU interpreter), the uniform
map, and the Box-Muller normals against scipy's normal distribution."""
import numpy as np
import pytest

from philox_ref import triton_philox


def test_philox_matches_triton_reference(orc):
    pytest.importorskip("triton")
    rng = np.random.default_rng(1234)
    cases = []
    for _ in range(6):
        seed = int(rng.integers(0, 2**63))
        ctrs = rng.integers(0, 2**32, size=(8, 4), dtype=np.uint64)
        ctrs[0] = 0
        ctrs[1] = [1, 0, 0, 0]
        cases.append([seed, ctrs.tolist()])
    cases.append([0, [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [7, 3, 1, 2 << 8 | 1], [1, 2, 3, 4]]])
    ref, why = triton_philox(cases)
    if ref is None:
        pytest.skip(why)
    for (seed, ctrs), want in zip(cases, ref):
        key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
        for ctr, w in zip(ctrs, want):
            got = orc.philox(ctr, key)
            assert got.tolist() == w, (seed, ctr)


def test_uniform_map_is_exact_float32_and_open_interval(orc):
    for r in [0, 1, 511, 512, 2**31, 2**32 - 1, 123456789]:
        u = orc.u01(r)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u
    assert orc.u01(0) == 2.0**-24
    assert orc.u01(2**32 - 1) == 1.0 - 2.0**-24


def test_normals_are_standard_normal(orc):
    stats = pytest.importorskip("scipy.stats")
    e = np.array([orc.normals5(7, i, 3) for i in range(40000)])
    for c in range(5):
        assert stats.kstest(e[:, c], "norm").pvalue > 1e-4
    assert abs(np.corrcoef(e[:, 0], e[:, 1])[0, 1]) < 0.03
    assert abs(np.corrcoef(e[:, 2], e[:, 4])[0, 1]) < 0.03
    # keyed by (seed, slot, frame): reproducible and frame-dependent
    assert np.array_equal(orc.normals5(7, 5, 3), orc.normals5(7, 5, 3))
    assert not np.array_equal(orc.normals5(7, 5, 3), orc.normals5(7, 5, 4))
    assert not np.array_equal(orc.normals5(7, 5, 3), orc.normals5(8, 5, 3))


def test_propagation_fields_and_uniforms(orc):
    """Six 21-bit fields of one 128-bit block, each mapped to an exact float32
    odd multiple of 2^-22; checked against Python's big-integer slicing."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        w = rng.integers(0, 2**32, size=4, dtype=np.uint64)
        big = int(w[0]) | int(w[1]) << 32 | int(w[2]) << 64 | int(w[3]) << 96
        want = [(big >> (21 * k)) & (2**21 - 1) for k in range(6)]
        assert orc.prop_fields(w).tolist() == want
    assert orc.prop_fields([0xFFFFFFFF] * 4).tolist() == [2**21 - 1] * 6
    assert orc.u21(0) == 2.0**-22
    assert orc.u21(2**21 - 1) == 1.0 - 2.0**-22
    for f in [0, 1, 12345, 2**20, 2**21 - 1]:
        u = orc.u21(f)
        assert float(np.float32(u)) == u and 0.0 < u < 1.0
