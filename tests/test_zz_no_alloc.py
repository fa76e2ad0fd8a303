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


RESET_SCRIPT = r"""
import ctypes as C, sys
import numpy as np
L = C.CDLL(sys.argv[1])
L.ppf_systematic_resample_noalloc.argtypes = [C.c_void_p, C.c_int64, C.c_uint64, C.c_uint32, C.c_int32,
                                              C.c_void_p, C.c_void_p]
n = 70001
rng = np.random.default_rng(3)
lw = (rng.standard_normal(n) * 3.0).astype(np.float32)

def once():
    # device buffers from the CUDA runtime the library is linked with
    d_lw, d_anc = C.c_void_p(), C.c_void_p()
    assert L.cudaMalloc(C.byref(d_lw), C.c_size_t(4 * n)) == 0
    assert L.cudaMalloc(C.byref(d_anc), C.c_size_t(4 * n)) == 0
    assert L.cudaMemcpy(d_lw, lw.ctypes.data_as(C.c_void_p), C.c_size_t(4 * n), 1) == 0
    assert L.ppf_systematic_resample_noalloc(d_lw, n, 9, 1, 5, d_anc, None) == 0
    out = np.zeros(n, dtype=np.int32)
    assert L.cudaMemcpy(out.ctypes.data_as(C.c_void_p), d_anc, C.c_size_t(4 * n), 2) == 0
    L.cudaFree(d_lw)
    L.cudaFree(d_anc)
    return out

a = once()
assert L.cudaDeviceReset() == 0   # ends this process's context only
b = once()                        # a new context: the scratch address is looked up again
assert np.array_equal(a, b) and np.all(np.diff(a) >= 0)
print("ok")
"""


def test_noalloc_after_device_reset():
    """After cudaDeviceReset the device has a new context; the entry point
    must look its scratch array up again rather than use the old address.
    Run in a child process that uses the CUDA runtime directly (no torch), so
    the reset touches no other test's state."""
    import os
    import subprocess
    import sys
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1310_5045_gb300 as ppf
    ppf.load()
    p = subprocess.run([sys.executable, "-c", RESET_SCRIPT, ppf.lib_path()], capture_output=True, text=True,
                       timeout=300, env=dict(os.environ, CUDA_VISIBLE_DEVICES=os.environ.get("CUDA_VISIBLE_DEVICES", "0")))
    assert p.returncode == 0 and p.stdout.strip().endswith("ok"), p.stdout[-500:] + p.stderr[-2000:]
