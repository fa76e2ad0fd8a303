"""The allocation-free systematic resampling entry point, for callers that
cannot call cudaMalloc (pre-planned serving / real-time loops, hosts whose
device memory belongs to another allocator).  Through the C ABI it must give
exactly the ancestors that the regular ppf_resample (PPF_SYSTEMATIC) gives
for the same log-weights, on consecutive calls that reuse its fixed scratch
array.  Collected last so a stop-at-first-failure run has run all other tests."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_resampling_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1310_5045_gb300 as ppf
    L = ppf.load()
    mv = synth.make_movie(W=128, H=128, K=3, seed=7)
    frames = torch.from_numpy(mv.frames).cuda()
    N = 50_003  # several tiles and a ragged tail
    m = ppf.Model(seed=11, filter_id=2)
    pf = ppf.ParticleFilter(m, N, group_size=4096)
    stream = torch.cuda.current_stream()
    for k in (1, 2):  # two calls in a row share (and must clear) the scratch array
        pf.step(frames[k - 1], k)
        st, _, _ = pf.get_particles()
        lw = st[5].contiguous()
        pf.resample(ppf.SYSTEMATIC)
        _, want, _ = pf.get_particles(state=False, anc=True)
        got = torch.full((N,), -1, dtype=torch.int32, device="cuda")
        rc = L.ppf_systematic_resample_noalloc(C.c_void_p(lw.data_ptr()), N, m.seed, m.filter_id, k,
                                               C.c_void_p(got.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == ppf.OK
        torch.cuda.synchronize()
        assert torch.equal(got, want), int((got != want).sum())
    # the python wrapper reaches the same symbol
    again = ppf._binding.systematic_resample_noalloc(lw, m.seed, m.filter_id, 2)
    assert torch.equal(again, want)
    # sizes beyond the scratch capacity are rejected, nothing is launched
    big = C.c_int64(16_777_217)
    assert L.ppf_systematic_resample_noalloc(C.c_void_p(lw.data_ptr()), big, 0, 0, 1,
                                             C.c_void_p(got.data_ptr()), None) == ppf.EINVAL
    pf.close()


def test_noalloc_degenerate_weights_give_identity():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1310_5045_gb300 as ppf
    n = 9000
    lw = torch.full((n,), float("nan"), device="cuda")
    out = ppf._binding.systematic_resample_noalloc(lw, 1, 0, 3)
    torch.cuda.synchronize()
    assert torch.equal(out.cpu(), torch.arange(n, dtype=torch.int32))
    lw = torch.zeros(n, device="cuda")
    lw[1234] = 5.0
    lw[:1000] = -float("inf")
    out = ppf._binding.systematic_resample_noalloc(lw, 1, 0, 4)
    torch.cuda.synchronize()
    # one particle 148x heavier than the rest: every ticket lands on a live particle
    a = out.cpu().numpy()
    assert np.all(a >= 1000) and np.all(np.diff(a) >= 0)
