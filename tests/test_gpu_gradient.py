"""GPU gradient of the log marginal likelihood estimate (ppf_loglik_grad,
forward-mode tangents) against the FP64 oracle's reverse mode on the same
stop-gradient path (the GPU's ancestors and patch anchors replayed), and
against central differences of that replayed objective (eps = 1e-3).

Tolerances: L is a sum of K log-evidences of float32 likelihoods (each 1e-5
relative, gpu_common), so 1e-5 relative; each derivative is a weighted mean of
float32 per-particle derivatives and must be within 1e-3 relative of the
central differences (the target), plus 1e-3 of the largest derivative scale
for components near zero."""
import math
import os

import numpy as np
import pytest

import oracle as orc
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1310_5045_gb300 as p
    p.load()
    return p


def setup_case(ppf, seed, N=4096, K=6):
    import torch
    from gpu_common import paired_models
    mv = synth.make_movie(W=64, H=56, K=K, sigma=1.5, amplitude=30.0, background=10.0, seed=seed,
                          start_frac=(0.4, 0.6))
    gm, om = paired_models(ppf, width=64, height=56, patch_radius=4, psf_sigma=1.5, amplitude=30.0,
                           background=10.0, sigma_m=0.5, sigma_I=0.0, seed=seed)
    fr = torch.from_numpy(mv.frames).cuda()
    return mv, gm, om, fr, N


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_oracle_and_differences(ppf, seed):
    mv, gm, om, fr, N = setup_case(ppf, seed)
    pf = ppf.ParticleFilter(gm, N, group_size=1024)
    theta = np.array([1.5, 30.0, 10.0, 0.5], dtype=np.float32).astype(np.float64)
    L, g, anc, anchors = pf.loglik_grad(fr, theta, return_path=True)
    a = anc.cpu().numpy()
    an = anchors.cpu().numpy()
    rc, Lo, go, _, _ = orc.grad_run(om, N, mv.frames, theta, a, an)
    assert rc == 0
    assert L == pytest.approx(Lo, rel=1e-5)
    scale = np.max(np.abs(go))
    assert np.all(np.abs(g - go) <= 1e-4 * np.abs(go) + 1e-5 * scale), (g, go)
    for c, h in enumerate([1e-3 * theta[0], 1e-3 * theta[1], 1e-3 * theta[2], 1e-3 * theta[3]]):
        tp, tm = theta.copy(), theta.copy()
        tp[c] += h
        tm[c] -= h
        fd = (orc.grad_run(om, N, mv.frames, tp, a, an)[1] - orc.grad_run(om, N, mv.frames, tm, a, an)[1]) / (2 * h)
        assert abs(g[c] - fd) <= 1e-3 * abs(fd) + 1e-3 * scale * 1e-2, (c, g[c], fd)
    pf.close()


def test_gradient_is_deterministic_and_autograd(ppf):
    import torch
    mv, gm, om, fr, N = setup_case(ppf, 2, N=2048, K=4)
    pf = ppf.ParticleFilter(gm, N, group_size=512)
    L1, g1 = pf.loglik_grad(fr)
    L2, g2 = pf.loglik_grad(fr)
    assert L1 == L2 and np.array_equal(g1, g2)
    th = torch.tensor([1.5, 30.0, 10.0, 0.5], dtype=torch.float64, requires_grad=True)
    out = ppf.log_marginal_likelihood(th, pf, fr)
    (gt,) = torch.autograd.grad(2.0 * out, th)
    assert out.item() == pytest.approx(L1, rel=1e-12)
    assert np.allclose(gt.numpy(), 2.0 * g1, rtol=1e-12)
    # after the gradient run the context holds weighted particles: resampling may follow
    pf.resample(ppf.SYSTEMATIC)
    pf.close()


def test_gradient_full_size(ppf):
    """The gradient workload in full, in the benchmark's launch configuration:
    N = 2^20 particles, 50 frames of 256 x 256, 9 x 9 patch, I0 = A, groups of
    4096.  The GPU's L and gradient against the oracle's reverse mode on the
    whole replayed stop-gradient path, and against central differences
    (eps = 1e-3 of each parameter) of the replayed objective."""
    import torch
    from gpu_common import paired_models
    free, _ = torch.cuda.mem_get_info()
    if free < 4 * 2**30:
        pytest.skip("needs ~4 GB of free device memory")
    orc.set_threads(os.cpu_count() or 1)
    gmv, gp = synth.preset("spot256_k50", seed=1)
    N = gp["N"]
    gm, om = paired_models(ppf, width=256, height=256, patch_radius=4, psf_sigma=1.5, amplitude=50.0,
                           background=10.0, sigma_m=0.5, sigma_v=0.1, sigma_I=0.0, seed=0)
    fr = torch.from_numpy(gmv.frames).cuda()
    pf = ppf.ParticleFilter(gm, N, group_size=4096)
    theta = np.array([1.5, 50.0, 10.0, 0.5], dtype=np.float32).astype(np.float64)
    L, g, anc, anchors = pf.loglik_grad(fr, theta, return_path=True)
    a = anc.cpu().numpy()
    an = anchors.cpu().numpy()
    del anc, anchors
    pf.close()
    rc, Lo, go, _, _ = orc.grad_run(om, N, gmv.frames, theta, a, an)
    assert rc == 0
    assert L == pytest.approx(Lo, rel=1e-5)
    scale = np.max(np.abs(go))
    assert np.all(np.abs(g - go) <= 1e-4 * np.abs(go) + 1e-5 * scale), (g, go)
    for c in range(4):
        h = 1e-3 * theta[c]
        tp, tm = theta.copy(), theta.copy()
        tp[c] += h
        tm[c] -= h
        fd = (orc.grad_run(om, N, gmv.frames, tp, a, an)[1] - orc.grad_run(om, N, gmv.frames, tm, a, an)[1]) / (2 * h)
        assert abs(g[c] - fd) <= 1e-3 * abs(fd) + 1e-5 * scale, (c, g[c], fd)
