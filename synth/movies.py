"""Synthetic single-spot fluorescence movies (Sec. 7: dynamics, eq. 3 appearance,
Poisson shot noise), seeded with numpy's PCG64.

Readings used here (all data-side only):
  * Pixel (i, j) is column i <-> x and row j <-> y, pixel centres at integer
    coordinates 0..W-1, and the PSF is point-sampled at the centres (eq. 3).
  * Truth dynamics per frame: x_k = x_{k-1} + v_{k-1} + sigma_m * e,
    v_k = 0.98 v_{k-1} + sigma_v * e' - kappa (x_{k-1} - centre), the spot
    intensity constant.  The weak pull kappa = (v0 / 0.3 W)^2 and the light
    damping keep long sequences in view with smooth turns; a reflection at a
    margin is the safety net.
  * SNR is the Poisson peak SNR I0 / sqrt(I0 + I_bg) (an amplitude ratio,
    "SNR 2 (6 dB)" in Sec. 7.3), so I0 solves I0^2 = SNR^2 (I0 + I_bg).
  * Frames are float32 photon counts.  Reduced-precision copies are made by the
    caller (counts <= 256 are exact in bf16, <= 2048 in fp16).
  * Streams: the seed's SeedSequence spawns one stream for the trajectory and
    one for the Poisson noise (in a batch, one pair per filter), each drawn
    frame after frame, so frame k is the same whatever the number of frames
    generated.
"""

from __future__ import annotations

import concurrent.futures
import dataclasses
import math
import os

import numpy as np


def amplitude_for_snr(snr: float, background: float) -> float:
    """Peak amplitude I0 with I0 / sqrt(I0 + bg) == snr (positive root)."""
    s2 = snr * snr
    return 0.5 * (s2 + math.sqrt(s2 * s2 + 4.0 * s2 * background))


@dataclasses.dataclass
class Movie:
    frames: np.ndarray        # (K, H, W) float32 photon counts
    truth: np.ndarray         # (K, 5) float64: x, y, vx, vy, I0 at each frame
    sigma: float              # PSF standard deviation [px]
    amplitude: float          # spot peak intensity I0
    background: float         # I_bg
    sigma_m: float            # truth position noise [px/frame]
    sigma_v: float            # truth velocity noise [px/frame^2]
    seed: int

    @property
    def K(self) -> int:
        return self.frames.shape[0]

    @property
    def H(self) -> int:
        return self.frames.shape[1]

    @property
    def W(self) -> int:
        return self.frames.shape[2]


def _render(W: int, H: int, x: float, y: float, amp: float, bg: float, sigma: float) -> np.ndarray:
    px = np.arange(W, dtype=np.float64)
    py = np.arange(H, dtype=np.float64)
    gx = np.exp(-((px - x) ** 2) / (2.0 * sigma * sigma))
    gy = np.exp(-((py - y) ** 2) / (2.0 * sigma * sigma))
    return bg + amp * np.outer(gy, gx)


def _trajectory(rng, K, W, H, start_lo, start_hi, v0, sigma_m, sigma_v, amp, margin):
    x = rng.uniform(start_lo[0], start_hi[0])
    y = rng.uniform(start_lo[1], start_hi[1])
    vx = rng.uniform(-v0, v0)
    vy = rng.uniform(-v0, v0)
    # a weak pull toward the image centre turns the spot smoothly, so long
    # sequences stay in view (swing of about 0.3 of the image for |v| <= v0)
    kx = (max(v0, 1e-3) / (0.3 * W)) ** 2
    ky = (max(v0, 1e-3) / (0.3 * H)) ** 2
    cx, cy = 0.5 * (W - 1), 0.5 * (H - 1)
    damp = 0.02  # keeps the velocity spread stationary (about sigma_v / sqrt(2 damp))
    truth = np.empty((K, 5), dtype=np.float64)
    for k in range(K):
        e = rng.standard_normal(4)
        nx = x + vx + sigma_m * e[0]
        ny = y + vy + sigma_m * e[1]
        vx = (1.0 - damp) * vx + sigma_v * e[2] - kx * (x - cx)
        vy = (1.0 - damp) * vy + sigma_v * e[3] - ky * (y - cy)
        # keep the spot inside the image (generator-side only)
        if nx < margin:
            nx, vx = 2 * margin - nx, abs(vx)
        if nx > W - 1 - margin:
            nx, vx = 2 * (W - 1 - margin) - nx, -abs(vx)
        if ny < margin:
            ny, vy = 2 * margin - ny, abs(vy)
        if ny > H - 1 - margin:
            ny, vy = 2 * (H - 1 - margin) - ny, -abs(vy)
        x, y = nx, ny
        truth[k] = (x, y, vx, vy, amp)
    return truth


def make_movie(
    W: int = 128,
    H: int = 128,
    K: int = 20,
    sigma: float = 1.5,
    amplitude: float = 50.0,
    background: float = 10.0,
    sigma_m: float = 0.5,
    sigma_v: float = 0.05,
    v0: float = 1.0,
    start_frac: tuple[float, float] = (0.25, 0.75),
    seed: int = 0,
    noise: bool = True,
) -> Movie:
    """One spot moving through K frames of W x H Poisson noise.  Frame k
    depends on the seed and k only, not on K."""
    traj_ss, noise_ss = np.random.SeedSequence(seed).spawn(2)
    rng = np.random.Generator(np.random.PCG64(traj_ss))
    lo = (start_frac[0] * W, start_frac[0] * H)
    hi = (start_frac[1] * W, start_frac[1] * H)
    margin = min(8.0, 0.1 * min(W, H))
    truth = _trajectory(rng, K, W, H, lo, hi, v0, sigma_m, sigma_v, amplitude, margin)
    frames = np.empty((K, H, W), dtype=np.float32)
    nrng = np.random.Generator(np.random.PCG64(noise_ss))
    for k in range(K):
        mu = _render(W, H, truth[k, 0], truth[k, 1], amplitude, background, sigma)
        frames[k] = nrng.poisson(mu) if noise else mu
    return Movie(frames, truth, sigma, amplitude, background, sigma_m, sigma_v, seed)


@dataclasses.dataclass
class MovieBatch:
    frames: np.ndarray        # (K, F, H, W) float32
    truth: np.ndarray         # (F, K, 5)
    sigma: np.ndarray         # (F,)
    amplitude: np.ndarray     # (F,)
    background: float
    n_particles: np.ndarray   # (F,) int64 particle counts, log-uniform
    seed: int


def make_movie_batch(
    F: int = 4096,
    W: int = 64,
    H: int = 64,
    K: int = 30,
    sigma_range=(1.0, 2.0),
    snr_range=(2.0, 8.0),
    background: float = 10.0,
    n_range=(256, 65536),
    sigma_m: float = 0.5,
    sigma_v: float = 0.05,
    seed: int = 0,
) -> MovieBatch:
    """F independent single-spot movies with uneven particle counts
    N_f = floor(exp(U[ln n_lo, ln n_hi])).  Filter f's frame k depends on the
    seed, f and k only, not on K."""
    par_ss, filt_ss = np.random.SeedSequence(seed).spawn(2)
    rng = np.random.Generator(np.random.PCG64(par_ss))
    sig = rng.uniform(*sigma_range, size=F)
    snr = rng.uniform(*snr_range, size=F)
    amp = np.array([amplitude_for_snr(s, background) for s in snr])
    n = np.floor(np.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]), size=F))).astype(np.int64)
    n = np.clip(n, n_range[0], n_range[1])
    frames = np.empty((K, F, H, W), dtype=np.float32)
    truth = np.empty((F, K, 5), dtype=np.float64)
    px = np.arange(W, dtype=np.float64)
    py = np.arange(H, dtype=np.float64)
    margin = min(8.0, 0.1 * min(W, H))
    noise = []
    for f, fss in enumerate(filt_ss.spawn(F)):
        traj_ss, noise_ss = fss.spawn(2)
        truth[f] = _trajectory(np.random.Generator(np.random.PCG64(traj_ss)), K, W, H, (0.25 * W, 0.25 * H),
                               (0.75 * W, 0.75 * H), 1.0, sigma_m, sigma_v, amp[f], margin)
        noise.append(noise_ss)

    def draw(f):
        s2 = 2.0 * sig[f] * sig[f]
        gx = np.exp(-((px[None, :] - truth[f, :, 0:1]) ** 2) / s2)   # (K, W)
        gy = np.exp(-((py[None, :] - truth[f, :, 1:2]) ** 2) / s2)   # (K, H)
        mu = background + amp[f] * gy[:, :, None] * gx[:, None, :]
        # one call draws the frames in order, frame 0 first
        frames[:, f] = np.random.Generator(np.random.PCG64(noise[f])).poisson(mu)

    # every filter has its own stream, so the draws may run on several threads
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(draw, range(F)))
    return MovieBatch(frames, truth, sig, amp, background, n, seed)


# Named workloads (sizes from the paper's experiment and its scaled variants).
PRESETS = {
    # 128x128, 20 frames, sigma 1.5, I0 50, bg 10, N = 16384, 9x9 patch
    "spot128_k20": dict(W=128, H=128, K=20, sigma=1.5, amplitude=50.0, background=10.0,
                        sigma_m=0.5, N=16384, r=4),
    # 512x512, 50 frames, sigma ~ U[1.2, 2.0], SNR ~ U[2, 8], N = 38e6, 11x11 patch
    "spot512_k50": dict(W=512, H=512, K=50, sigma=None, amplitude=None, background=10.0,
                        sigma_m=0.5, N=38_000_000, r=5),
    # 256x256, 50 frames, gradient workload, N = 2^20, 9x9 patch
    "spot256_k50": dict(W=256, H=256, K=50, sigma=1.5, amplitude=50.0, background=10.0,
                        sigma_m=0.5, N=1 << 20, r=4),
}


def preset(name: str, seed: int = 0, K: int | None = None) -> tuple[Movie, dict]:
    """Build the named workload's movie; returns (movie, filter settings)."""
    p = dict(PRESETS[name])
    rng = np.random.Generator(np.random.PCG64(10_000 + seed))
    if p["sigma"] is None:
        p["sigma"] = float(rng.uniform(1.2, 2.0))
    if p["amplitude"] is None:
        p["amplitude"] = amplitude_for_snr(float(rng.uniform(2.0, 8.0)), p["background"])
    kk = p["K"] if K is None else K
    mv = make_movie(W=p["W"], H=p["H"], K=kk, sigma=p["sigma"], amplitude=p["amplitude"],
                    background=p["background"], sigma_m=p["sigma_m"], seed=seed)
    return mv, p
