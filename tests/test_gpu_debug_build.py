"""The debug build (PPF_DEBUG=1 loads libppf_debug.so, compiled with
-DPPF_DEBUG): every scattered store of the resampling kernels and every patch
window of the step kernels is checked on the device before the access, a
failed check setting the internal-error flag (PPF_EINVAL from ppf_estimate /
ppf_batch_estimates) instead of faulting.  A subset of the GPU parity tests
runs against it in a child process: every resampling scheme at tile-crossing
and ragged sizes, ARNA, pcSIR, odd frame sizes with border particles, a single
particle, particles outside the image and batched filters."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_under_the_debug_build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, PPF_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", "import paper_1310_5045_gb300 as p; p.load(); print(p.lib_path())"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and r.stdout.strip().endswith("libppf_debug.so"), r.stdout + r.stderr
    sel = ("lockstep_frames or schemes_in_sequence or two_stage or tiny_and_ragged or arna "
           "or piecewise_constant_likelihood or odd_frame or single_particle or outside_image or equals_single "
           "or batch_lockstep")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu",
                        os.path.join("tests", "test_gpu_parity.py"), os.path.join("tests", "test_gpu_batch.py"),
                        "-k", sel], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
