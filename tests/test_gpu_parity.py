"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs (tolerances derived in tests/gpu_common.py)."""
import dataclasses
import math

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


@pytest.fixture(scope="module")
def movie():
    return synth.make_movie(W=128, H=128, K=6, sigma=1.5, amplitude=50.0, background=10.0, seed=0)


def gpu_frames(movie, dtype=None):
    import torch
    t = torch.from_numpy(movie.frames).cuda()
    return t if dtype is None else t.to(dtype)


def test_init_matches_oracle(ppf):
    from gpu_common import paired_models
    gm, om = paired_models(ppf, width=100, height=77, v0_max=0.75, amplitude=20.0)
    N = 10001
    pf = ppf.ParticleFilter(gm, N, group_size=1000)
    st, anc, lwp = pf.get_particles(state=True, anc=True, lw_prev=True)
    ref = orc.init(om, N)
    got = st.cpu().double().numpy()
    assert np.allclose(got, ref, rtol=2e-7, atol=1e-7)
    assert np.array_equal(anc.cpu().numpy(), np.arange(N))
    assert np.all(lwp.cpu().numpy() == 0.0)
    pf.close()


@pytest.mark.parametrize("scheme", [orc.SYSTEMATIC, orc.RPA_GS, orc.RPA_SGS, orc.RPA_LGS, orc.RNA,
                                    orc.RPA2_GS, orc.RPA2_SGS, orc.RPA2_LGS])
@pytest.mark.parametrize("N,gs", [(16384, 4096), (10000, 777)])
def test_lockstep_frames(ppf, movie, scheme, N, gs):
    from gpu_common import lockstep, paired_models
    gm, om = paired_models(ppf, seed=3)
    pf = ppf.ParticleFilter(gm, N, group_size=gs)
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), scheme, K=6, alpha=0.25)
    pf.close()


@pytest.mark.parametrize("N,gs", [(16384, 4096), (20000, 1500), (10000, 777), (9001, 5000), (40000, 20000),
                                  (50001, 12345), (200000, 4000)])
def test_rpa_schemes_in_sequence(ppf, movie, N, gs):
    """GS and SGS write every group's kept tickets straight to its balanced
    slots and copy only the links; LGS leaves unequal groups, so the GS and
    SGS frames after it start from tiles crossed by several groups of
    different sizes (the per-tile table, and the per-ticket lookup where more
    than five groups cross a tile).  Groups above two tiles (40000 / 20000,
    50001 / 12345, and those LGS grows) are drawn by the two-stage fill one
    tile per block, and groups with more than 8192 offspring (the
    concentrated clouds at N = 200000) one run of 8192 tickets per block."""
    from gpu_common import lockstep, paired_models
    gm, om = paired_models(ppf, seed=5)
    pf = ppf.ParticleFilter(gm, N, group_size=gs)
    seq = [orc.RPA_LGS, orc.RPA_GS, orc.RPA_LGS, orc.RPA_LGS, orc.RPA_SGS, orc.RPA2_LGS]
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), seq, K=6)
    seq = [orc.RPA_LGS, orc.RPA2_GS, orc.RPA2_LGS, orc.RPA2_SGS, orc.RPA_GS, orc.SYSTEMATIC]
    log = []
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), seq, K=6, log=log)
    if N == 200000:  # the run split is exercised: some frame gives one group > 8192 offspring
        assert max(e[2] for e in log if e[0] == "offspring") > 8192
    pf.close()


@pytest.mark.parametrize("scheme", [orc.RPA2_GS, orc.RPA2_SGS, orc.RPA2_LGS])
def test_two_stage_large_groups_with_heavy_tiles(ppf, movie, scheme):
    """Groups of 50000 particles (above two tiles) are drawn one tile part per
    block, and a tile part with more than 8192 offspring (the concentrated
    clouds of this movie put several times that in one tile) one run of 8192
    tickets per block."""
    from gpu_common import lockstep, paired_models
    gm, om = paired_models(ppf, seed=7)
    pf = ppf.ParticleFilter(gm, 200000, group_size=50000)
    log = []
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), scheme, K=5, log=log)
    assert max(e[2] for e in log if e[0] == "tile offspring") > 8192
    pf.close()


@pytest.mark.parametrize("scheme", [orc.SYSTEMATIC, orc.RPA_SGS, orc.RNA, orc.RPA2_GS, orc.ARNA])
def test_ess_gated_resampling(ppf, scheme):
    """Alg. 1's N_eff test on the device: with sigma_xi^2 = 2000 and a
    threshold of 4000 (N = 16384) the filter keeps the particles at some
    frames and resamples at the others."""
    from gpu_common import lockstep, paired_models
    mv = synth.make_movie(W=128, H=128, K=8, sigma=1.5, amplitude=50.0, background=10.0, seed=0)
    gm, om = paired_models(ppf, seed=3, sigma_xi=math.sqrt(2000.0))
    pf = ppf.ParticleFilter(gm, 16384, group_size=4096)
    log = []
    lockstep(pf, gm, om, mv.frames, gpu_frames(mv), scheme, K=8, alpha=0.25, log=log, ess_threshold=4000.0)
    kept = [e[2] for e in log if e[0] == "kept"]
    assert any(kept) and not all(kept), kept
    pf.close()


@pytest.mark.parametrize("scheme", [orc.RPA_GS, orc.RPA_LGS, orc.RPA2_SGS])
def test_rpa_at_the_group_limit(ppf, movie, scheme):
    """The RPA schedules at their largest group count, G = 16384 groups of 40
    particles (one block sorts and merges every sender and receiver), and one
    group more is rejected."""
    from gpu_common import lockstep, paired_models
    gm, om = paired_models(ppf, seed=9)
    pf = ppf.ParticleFilter(gm, 16384 * 40, group_size=40)
    assert len(pf.groups()) == 16385
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), scheme, K=2)
    pf.close()
    pf = ppf.ParticleFilter(gm, 16385 * 40, group_size=40)
    pf.step(gpu_frames(movie)[0], 1)
    with pytest.raises(ppf.PPFError) as e:
        pf.resample(scheme)
    assert e.value.status == ppf.EINVAL
    pf.resample(ppf.SYSTEMATIC)  # the other schemes have no group limit
    pf.close()


@pytest.mark.parametrize("scheme", [orc.SYSTEMATIC, orc.RNA])
@pytest.mark.parametrize("r", [2, 4, 8])
def test_piecewise_constant_likelihood(ppf, movie, scheme, r):
    """pcSIR: every particle's likelihood is looked up in the per-frame map of
    cell-centre patch sums; lockstep against the oracle's pcSIR reading."""
    from gpu_common import lockstep, paired_models
    gm, om = paired_models(ppf, seed=13, patch_radius=r, likelihood=1)
    pf = ppf.ParticleFilter(gm, 12000, group_size=3000)
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), scheme, K=4, alpha=0.2)
    pf.close()


def test_piecewise_constant_likelihood_is_rejected_where_unsupported(ppf, movie):
    from gpu_common import paired_models
    gm, _ = paired_models(ppf, seed=13, likelihood=1)
    pf = ppf.ParticleFilter(gm, 1000, group_size=1000)
    with pytest.raises(ppf.PPFError) as e:
        pf.loglik_grad(gpu_frames(movie)[:2])
    assert e.value.status == ppf.EINVAL
    pf.close()
    with pytest.raises(ppf.PPFError):
        ppf.BatchFilter([gm, gm], [100, 100])
    bad = paired_models(ppf, seed=13, likelihood=2)[0]
    with pytest.raises(ppf.PPFError):
        ppf.ParticleFilter(bad, 100, group_size=100)


@pytest.mark.parametrize("r", [0, 1, 5, 8])
def test_patch_radius_and_ragged_tile(ppf, movie, r):
    from gpu_common import lockstep, paired_models
    gm, om = paired_models(ppf, patch_radius=r, seed=5)
    pf = ppf.ParticleFilter(gm, 4097, group_size=4097)
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), orc.SYSTEMATIC, K=3)
    pf.close()


def test_single_particle(ppf, movie):
    from gpu_common import lockstep, paired_models
    gm, om = paired_models(ppf, seed=1)
    pf = ppf.ParticleFilter(gm, 1, group_size=1)
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), orc.RPA_LGS, K=3)
    pf.close()


@pytest.mark.parametrize("N,gs", [(1, 1), (2, 1), (3, 2), (5, 5), (33, 4), (4097, 4097), (4097, 1)])
def test_tiny_and_ragged_layouts_every_scheme(ppf, movie, N, gs):
    """Degenerate layouts for every scheme: one particle, one particle per
    group, one group, a ragged last group, a group one past a tile, and 4097
    groups of one particle (more group starts in a tile than the routing
    table holds)."""
    from gpu_common import lockstep, paired_models
    gm, om = paired_models(ppf, seed=11)
    seq = [orc.SYSTEMATIC, orc.RPA_GS, orc.RPA_SGS, orc.RPA_LGS, orc.RNA, orc.RPA2_GS, orc.RPA2_SGS,
           orc.RPA2_LGS, orc.ARNA]
    pf = ppf.ParticleFilter(gm, N, group_size=gs)
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), seq[:6], K=6)
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), (seq[6:] + seq)[:6], K=6)
    pf.close()


@pytest.mark.parametrize("dtype_name", ["bfloat16", "float16"])
def test_reduced_precision_frames(ppf, movie, dtype_name):
    """Frames stored in BF16 / FP16; the oracle sees the same stored values."""
    import torch
    from gpu_common import lockstep, paired_models
    dt = getattr(torch, dtype_name)
    gm, om = paired_models(ppf, seed=2, frame_dtype=ppf.BF16 if dtype_name == "bfloat16" else ppf.F16)
    fr = gpu_frames(movie, dt)
    stored = fr.float().cpu().numpy()
    pf = ppf.ParticleFilter(gm, 8192, group_size=2048)
    lockstep(pf, gm, om, stored, fr, orc.SYSTEMATIC, K=4)
    pf.close()


def test_sis_without_resampling_carries_weights(ppf, movie):
    from gpu_common import lockstep, paired_models
    gm, om = paired_models(ppf, seed=4)
    pf = ppf.ParticleFilter(gm, 3000, group_size=1000)
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), None, K=3)
    pf.close()


def test_particles_outside_image(ppf, movie):
    """Particles whose patch leaves the image: partial patches and empty sums,
    and non-finite and huge finite states.  (The huge values share a sign: a
    posterior mean over weighted states of +1e30 and -1e30 cancels exactly in
    FP64 but not in float32, and says nothing about the path.)"""
    import torch
    from gpu_common import lockstep, paired_models
    gm, om = paired_models(ppf, seed=6, sigma_m=0.0, sigma_v=0.0, sigma_I=0.0)
    N = 2048
    rng = np.random.default_rng(0)
    st = np.zeros((6, N), dtype=np.float32)
    st[0] = rng.uniform(-14, 142, N)
    st[1] = rng.uniform(-14, 142, N)
    st[4] = rng.uniform(10, 80, N)
    st[0, :4] = [np.nan, np.inf, 1e30, 3e29]
    pf = ppf.ParticleFilter(gm, N, group_size=512)
    pf.set_particles(torch.from_numpy(st))
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), orc.SYSTEMATIC, K=2)
    pf.close()


@pytest.mark.parametrize("r", [1, 3, 6])
def test_odd_frame_sizes_and_borders(ppf, r):
    """Odd frame widths and heights (the pixel-pair rows then have odd
    lengths) with particles all over and around the image."""
    import torch
    from gpu_common import lockstep, paired_models
    W, H = 97, 61
    mv = synth.make_movie(W=W, H=H, K=3, sigma=1.3, amplitude=40.0, background=10.0, seed=4)
    gm, om = paired_models(ppf, width=W, height=H, patch_radius=r, seed=12, psf_sigma=1.3, amplitude=40.0)
    N = 6000
    rng = np.random.default_rng(r)
    st = np.zeros((6, N), dtype=np.float32)
    st[0] = rng.uniform(-2 * r - 3, W + 2 * r + 3, N)
    st[1] = rng.uniform(-2 * r - 3, H + 2 * r + 3, N)
    st[2:4] = rng.normal(0.0, 0.5, (2, N))
    st[4] = rng.uniform(10, 70, N)
    pf = ppf.ParticleFilter(gm, N, group_size=1000)
    pf.set_particles(torch.from_numpy(st))
    lockstep(pf, gm, om, mv.frames, gpu_frames(mv), orc.RPA_SGS, K=3)
    pf.close()


def test_degenerate_weights_keep_particles(ppf, movie):
    import torch
    from gpu_common import paired_models
    gm, om = paired_models(ppf)
    N = 5000
    pf = ppf.ParticleFilter(gm, N, group_size=1000)
    st, _, _ = pf.get_particles()
    pf.set_particles(st, lw_prev=torch.full((N,), float("nan")))
    pf.step(gpu_frames(movie)[0], 1)
    e = pf.estimate()
    assert e.status == ppf.EDEGENERATE
    before, _, _ = pf.get_particles()
    pf.resample(ppf.SYSTEMATIC)
    e = pf.estimate()
    assert e.status == ppf.EDEGENERATE
    _, anc, lwp = pf.get_particles(state=False, anc=True, lw_prev=True)
    assert np.array_equal(anc.cpu().numpy(), np.arange(N))
    assert torch.isnan(lwp).all()
    assert pf.estimate().status == ppf.OK  # flags are cleared once reported
    pf.close()


def test_step_host_matches_device_frames(ppf, movie):
    """Host frames (page-locked, double-buffered copies overlapping the
    previous frame; then one pageable frame) give bit-identical particles to
    device frames."""
    import torch
    from gpu_common import paired_models
    gm, _ = paired_models(ppf, seed=6)
    fr = gpu_frames(movie)
    host = torch.from_numpy(movie.frames).pin_memory()
    a = ppf.ParticleFilter(gm, 20000, group_size=4096)
    b = ppf.ParticleFilter(gm, 20000, group_size=4096)
    for k in range(1, 6):
        a.step_host(host[k - 1] if k < 5 else torch.from_numpy(movie.frames[k - 1].copy()), k)
        a.resample(ppf.SYSTEMATIC)
        b.step(fr[k - 1], k)
        b.resample(ppf.SYSTEMATIC)
    sa, aa, _ = a.get_particles(state=True, anc=True)
    sb, ab, _ = b.get_particles(state=True, anc=True)
    assert torch.equal(sa, sb) and torch.equal(aa, ab)
    a.close()
    b.close()


def test_checkpoint_and_resume(ppf, movie):
    """A run snapshotted after LGS left the groups unequal (particles, pending
    ancestors and starting weights, group layout, ARNA ring) resumes in a new
    context bit for bit: LGS, RNA, ARNA, then systematic frames."""
    import torch
    from gpu_common import paired_models
    gm, _ = paired_models(ppf, seed=8)
    fr = gpu_frames(movie)
    a = ppf.ParticleFilter(gm, 30000, group_size=1000)
    for k in (1, 2):
        a.step(fr[k - 1], k)
        a.resample(ppf.RPA_LGS)
    st, anc, lwp = a.get_particles(state=True, anc=True, lw_prev=True)
    goff = a.groups()
    assert len(set(np.diff(goff).tolist())) > 1  # LGS left the groups unequal
    a.set_ring(np.random.default_rng(0).permutation(30))  # an ARNA ring other than the identity
    ring = a.ring()
    b = ppf.ParticleFilter(gm, 30000, group_size=1000)
    b.set_particles(st, anc, lwp)
    b.set_groups(goff)
    b.set_ring(ring)
    for k, sch in ((3, ppf.RPA_LGS), (4, ppf.RNA), (5, ppf.ARNA), (6, ppf.SYSTEMATIC)):
        for f in (a, b):
            f.step(fr[k - 1], k)
            f.resample(sch, 0.3)
        sa, aa, la = a.get_particles(state=True, anc=True, lw_prev=True)
        sb, ab, lb = b.get_particles(state=True, anc=True, lw_prev=True)
        assert torch.equal(sa, sb) and torch.equal(aa, ab) and torch.equal(la, lb), k
        assert np.array_equal(a.groups(), b.groups())
        assert np.array_equal(a.ring(), b.ring())
    with pytest.raises(ppf.PPFError):
        b.set_groups(np.zeros(len(goff), dtype=np.int64))  # does not end at N
    a.close()
    b.close()


@pytest.mark.parametrize("N,gs", [(16384, 1024), (10000, 777)])
def test_arna_lockstep_with_a_lost_object(ppf, N, gs):
    """ARNA frame by frame against the oracle on a movie whose spot vanishes
    for two frames: the exchange ratio follows the involved groups, the ring
    is redrawn on the frames the object is lost (negative log-evidence) and
    kept otherwise; ancestors, weights, ring and counts bit-exact."""
    from gpu_common import lockstep, paired_models
    mv = synth.make_movie(W=128, H=128, K=8, sigma=1.5, amplitude=50.0, background=10.0, seed=4)
    blank = synth.make_movie(W=128, H=128, K=8, sigma=1.5, amplitude=0.0, background=10.0, seed=5)
    frames = mv.frames.copy()
    frames[3:5] = blank.frames[3:5]
    gm, om = paired_models(ppf, seed=6)
    pf = ppf.ParticleFilter(gm, N, group_size=gs)
    log = []
    lockstep(pf, gm, om, frames, gpu_frames(dataclasses.replace(mv, frames=frames)), orc.ARNA, K=8, alpha=0.5,
             log=log)
    lost = [e[2] for e in log if isinstance(e, tuple) and e[0] == "lost"]
    assert any(lost) and not all(lost)
    pf.close()


def test_arna_ring_accessors(ppf, movie):
    from gpu_common import paired_models
    gm, _ = paired_models(ppf, seed=1)
    pf = ppf.ParticleFilter(gm, 8000, group_size=1000)
    assert np.array_equal(pf.ring(), np.arange(8))
    pf.set_ring([3, 1, 2, 0, 7, 6, 5, 4])
    assert np.array_equal(pf.ring(), [3, 1, 2, 0, 7, 6, 5, 4])
    for bad in ([0, 1, 2, 3, 4, 5, 6, 6], [0, 1, 2, 3, 4, 5, 6, 8], [-1, 1, 2, 3, 4, 5, 6, 7]):
        with pytest.raises(ppf.PPFError):
            pf.set_ring(bad)
    assert np.array_equal(pf.ring(), [3, 1, 2, 0, 7, 6, 5, 4])
    pf.set_groups(pf.groups())  # a new layout starts from the identity ring
    assert np.array_equal(pf.ring(), np.arange(8))
    with pytest.raises(ppf.PPFError):
        pf.resample(ppf.ARNA, 1.5)   # ratio outside [0, 1]
    pf.close()


def test_injected_host_faults_leave_the_context_usable(ppf, movie, monkeypatch):
    """Host-side fault injection (no GPU fault): a failed launch is reported
    as PPF_ECUDA with its message, a bounded-wait timeout as PPF_ETIMEOUT from
    ppf_estimate; without the fault the same context steps and estimates."""
    from gpu_common import paired_models
    gm, _ = paired_models(ppf, seed=2)
    fr = gpu_frames(movie)
    pf = ppf.ParticleFilter(gm, 4096, group_size=1024)
    monkeypatch.setenv("PPF_FAULT", "launch")
    with pytest.raises(ppf.PPFError) as err:
        pf.step(fr[0], 1)
    assert err.value.status == ppf.ECUDA and "injected launch failure" in str(err.value)
    monkeypatch.delenv("PPF_FAULT")
    pf.step(fr[0], 1)
    monkeypatch.setenv("PPF_FAULT", "timeout")
    e = pf.estimate()
    assert e.status == ppf.ETIMEOUT
    assert e.status_flags & 2
    with pytest.raises(ppf.PPFError):
        pf.estimate(raise_on_flags=True)
    monkeypatch.delenv("PPF_FAULT")
    e = pf.estimate()
    assert e.status == 0 and e.status_flags == 0 and math.isfinite(e.log_evidence)
    pf.resample(ppf.SYSTEMATIC)
    pf.step(fr[1], 2)
    assert pf.estimate().status == 0
    pf.close()


def test_estimate_async_matches_estimate(ppf, movie):
    """Queued estimate copies (one per frame, read after the last frame) equal
    the synchronous estimates of the same frames."""
    import torch
    from gpu_common import paired_models
    gm, _ = paired_models(ppf, seed=2)
    fr = gpu_frames(movie)
    a = ppf.ParticleFilter(gm, 5000, group_size=1000)
    b = ppf.ParticleFilter(gm, 5000, group_size=1000)
    slots = torch.empty((4, ppf.Estimate.nbytes()), dtype=torch.uint8).pin_memory()
    want = []
    for k in range(1, 5):
        a.step(fr[k - 1], k)
        a.resample(ppf.RPA_SGS)
        a.estimate_async(slots[k - 1])
        b.step(fr[k - 1], k)
        b.resample(ppf.RPA_SGS)
        want.append(b.estimate())
    a.stream.synchronize()
    for k in range(4):
        got = ppf.Estimate.from_buffer(slots[k])
        w = want[k]
        assert got.frame == w.frame == k + 1
        assert got.mean == w.mean and got.ess == w.ess and got.log_evidence == w.log_evidence
        assert (got.links, got.moved, got.max_group, got.min_group) == (w.links, w.moved, w.max_group, w.min_group)
    a.close()
    b.close()


def test_state_errors(ppf):
    from gpu_common import paired_models
    gm, _ = paired_models(ppf)
    pf = ppf.ParticleFilter(gm, 100, group_size=10)
    with pytest.raises(ppf.PPFError) as e:
        pf.resample(ppf.SYSTEMATIC)
    assert e.value.status == ppf.ESTATE
    with pytest.raises(ppf.PPFError) as e:
        pf.estimate(raise_on_flags=True)
    assert e.value.status == ppf.ESTATE
    pf.close()


def test_free_running_tracks_the_spot(ppf):
    """End to end (no lockstep): the GPU filter tracks the synthetic spot."""
    import torch
    from gpu_common import paired_models
    mv = synth.make_movie(W=128, H=128, K=20, sigma=1.5, amplitude=50.0, background=10.0, seed=0)
    gm, om = paired_models(ppf, seed=0, sigma_xi=math.sqrt(200.0))
    fr = torch.from_numpy(mv.frames).cuda()
    pf = ppf.ParticleFilter(gm, 16384, group_size=4096)
    est = []
    for k in range(1, 21):
        pf.step(fr[k - 1], k)
        est.append(pf.estimate().mean)
        pf.resample(ppf.SYSTEMATIC)
    est = np.array(est)
    err = est[5:, :2] - mv.truth[5:, :2]
    assert np.sqrt((err ** 2).sum(1).mean()) < 0.5
    pf.close()


# ------------------------------------------------------------ likelihood paths
def _path_run(ppf, gm, N, gs, frames, path, schemes, init=None):
    """Frames through a context on one likelihood path; every output per frame."""
    import torch
    pf = ppf.ParticleFilter(gm, N, group_size=gs)
    pf.set_likelihood_path(path)
    if init is not None:
        pf.set_particles(torch.from_numpy(init))
    out = []
    for k in range(1, frames.shape[0] + 1):
        pf.step(frames[k - 1], k)
        e = pf.estimate()
        st, _, _ = pf.get_particles()
        binned = pf.last_step_binned()
        pf.resample(schemes[(k - 1) % len(schemes)], 0.25)
        _, anc, lwp = pf.get_particles(state=False, anc=True, lw_prev=True)
        out.append((st.cpu().numpy(), anc.cpu().numpy(), lwp.cpu().numpy(), e.mean, e.log_evidence, e.ess,
                    e.max_log_weight, binned))
    pf.close()
    return out


def _same(a, b):
    for k, ((sa, aa, la, ma, le_a, ea, xa, ba), (sb, ab, lb, mb, le_b, eb, xb, bb)) in enumerate(zip(a, b)):
        assert np.array_equal(sa, sb, equal_nan=True), k
        assert np.array_equal(aa, ab) and np.array_equal(la, lb, equal_nan=True), k
        assert np.array_equal(np.array([*ma, le_a, ea, xa]), np.array([*mb, le_b, eb, xb]), equal_nan=True), k


@pytest.mark.parametrize("r", [0, 1, 4, 5, 8])
def test_binned_path_equals_direct_path(ppf, movie, r):
    """The binned likelihood path (particles binned by image tile, each tile's
    window staged in shared memory by the tensor-memory accelerator) and the
    direct path give the same bits for every output of the step: state,
    log-weights, ancestors, posterior mean, log-evidence, N_eff.  Frame 1 is
    the prior draw, spread over the whole frame."""
    from gpu_common import paired_models
    gm, _ = paired_models(ppf, seed=21, patch_radius=r)
    fr = gpu_frames(movie)[:4]
    schemes = [ppf.SYSTEMATIC, ppf.RPA_SGS, ppf.RNA, ppf.ARNA]
    d = _path_run(ppf, gm, 20011, 2000, fr, ppf.PATH_DIRECT, schemes)
    b = _path_run(ppf, gm, 20011, 2000, fr, ppf.PATH_BINNED, schemes)
    assert not any(x[7] for x in d) and all(x[7] for x in b)
    _same(d, b)


def test_binned_path_odd_frames_borders_and_nonfinite(ppf):
    """Both paths on a 97 x 61 frame with particles all around and outside
    the borders, and non-finite and huge states (the bin of particles with no
    patch sum)."""
    import torch
    from gpu_common import paired_models
    W, H = 97, 61
    mv = synth.make_movie(W=W, H=H, K=3, sigma=1.3, amplitude=40.0, background=10.0, seed=4)
    gm, _ = paired_models(ppf, width=W, height=H, patch_radius=3, seed=12, psf_sigma=1.3, amplitude=40.0)
    N = 7001
    rng = np.random.default_rng(3)
    st = np.zeros((6, N), dtype=np.float32)
    st[0] = rng.uniform(-12, W + 12, N)
    st[1] = rng.uniform(-12, H + 12, N)
    st[2:4] = rng.normal(0.0, 0.5, (2, N))
    st[4] = rng.uniform(10, 70, N)
    st[0, :4] = [np.nan, np.inf, 1e30, -3.0]
    st[4, 4] = np.nan
    fr = torch.from_numpy(mv.frames).cuda()
    schemes = [ppf.SYSTEMATIC, ppf.RPA_LGS]
    d = _path_run(ppf, gm, N, 1000, fr, ppf.PATH_DIRECT, schemes, init=st)
    b = _path_run(ppf, gm, N, 1000, fr, ppf.PATH_BINNED, schemes, init=st)
    _same(d, b)


@pytest.mark.parametrize("scheme", [orc.SYSTEMATIC, orc.RPA_SGS, orc.RNA])
def test_binned_path_lockstep(ppf, movie, scheme):
    """The binned path frame by frame against the oracle."""
    from gpu_common import lockstep, paired_models
    gm, om = paired_models(ppf, seed=3)
    pf = ppf.ParticleFilter(gm, 16384, group_size=4096)
    pf.set_likelihood_path(ppf.PATH_BINNED)
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), scheme, K=4, alpha=0.25)
    pf.close()


def test_automatic_path_choice(ppf):
    """Chosen on the device: the prior draw (spread over the frame) is binned;
    the systematic draw after it (N_eff far below N / 64) collapses the cloud
    onto the spot, so the next step is direct already.  Without resampling
    (SIS) or with RNA's local draws the cloud stays spread, and so does the
    binned path."""
    from gpu_common import paired_models
    mv = synth.make_movie(W=512, H=512, K=6, sigma=1.5, amplitude=50.0, background=10.0, seed=2)
    gm, _ = paired_models(ppf, width=512, height=512, patch_radius=5, seed=2)
    fr = gpu_frames(mv)
    for scheme, want in [(ppf.SYSTEMATIC, [True, False]), (ppf.RPA_SGS, [True, False]), (None, [True, True]),
                         (ppf.RNA, [True, True])]:
        pf = ppf.ParticleFilter(gm, 200_000, group_size=4096)
        seen = []
        for k in range(1, 7 if scheme == ppf.SYSTEMATIC else 3):
            pf.step(fr[k - 1], k)
            seen.append(pf.last_step_binned())
            if scheme is not None:
                pf.resample(scheme, 0.1)
        assert seen[:2] == want, (scheme, seen)
        if scheme == ppf.SYSTEMATIC:
            assert not any(seen[1:]), seen
        pf.close()
    # a fixed path ignores both the tally and the concentrating draw
    for path, want in [(ppf.PATH_BINNED, True), (ppf.PATH_DIRECT, False)]:
        pf = ppf.ParticleFilter(gm, 200_000, group_size=4096)
        pf.set_likelihood_path(path)
        seen = []
        for k in range(1, 4):
            pf.step(fr[k - 1], k)
            seen.append(pf.last_step_binned())
            pf.resample(ppf.SYSTEMATIC)
        assert seen == [want] * 3, (path, seen)
        pf.close()
    pf = ppf.ParticleFilter(gm, 200_000, group_size=4096)
    with pytest.raises(ppf.PPFError):
        pf.set_likelihood_path(7)
    pf.close()
    pc, _ = paired_models(ppf, seed=2, likelihood=1)
    p2 = ppf.ParticleFilter(pc, 1000, group_size=1000)
    with pytest.raises(ppf.PPFError) as e:
        p2.set_likelihood_path(ppf.PATH_BINNED)
    assert e.value.status == ppf.EINVAL
    p2.set_likelihood_path(ppf.PATH_DIRECT)
    p2.close()


@pytest.mark.parametrize("path", ["direct", "binned"])
def test_arna_unequal_groups_and_permuted_ring(ppf, movie, path):
    """ARNA on an LGS-like layout of unequal groups installed with
    ppf_set_groups and a permuted ring installed with ppf_set_ring, in
    lockstep against the oracle: the involved test against each group's own
    size, the migrant count from the smallest group, the exchange along the
    permuted ring; ancestors, weights, ring and counts bit-exact."""
    from gpu_common import lockstep, paired_models
    gm, om = paired_models(ppf, seed=9)
    sizes = np.array([2500, 600, 1900, 1300, 3700, 2000, 4384])
    N = int(sizes.sum())
    pf = ppf.ParticleFilter(gm, N, group_size=2400)  # ceil(16384 / 2400) = 7 groups
    G = len(pf.groups()) - 1
    assert G == len(sizes)
    pf.set_groups(np.concatenate([[0], np.cumsum(sizes)]))
    pf.set_ring(np.array([3, 0, 6, 4, 1, 5, 2], dtype=np.int32))
    pf.set_likelihood_path(ppf.PATH_DIRECT if path == "direct" else ppf.PATH_BINNED)
    log = []
    lockstep(pf, gm, om, movie.frames, gpu_frames(movie), orc.ARNA, K=4, alpha=0.5, log=log)
    e = pf.estimate()
    assert e.moved > 0 and e.min_group == 600 and e.max_group == 4384
    pf.close()
