"""Seeded synthetic frames shaped like the workloads of arXiv 2310.08770.

This module only *generates inputs*: a Gaussian spot integrated over each
pixel, with Poisson shot noise, at exactly known displacements (Sec. IV, the
synthetic-data recipe). It holds none of the tracking arithmetic, so the FP64
oracle and the CUDA path can both be fed from it without sharing any of the
method's code.

Conventions: images are H rows x W columns, row-major, x = column index.
Pixel (y, x) has its centre at integer coordinates (y, x). A frame whose spot
sits at (y0 + dy, x0 + dx) while the reference spot sits at (y0, x0) has the
displacement d = (dx, dy): frame(r) ~ ref(r - d).

Draw order for every workload: parameters, then trajectory / shifts, then the
noise of each frame in frame order, all from one ``numpy.random.default_rng``
(PCG64) stream seeded by ``seed``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import erf

__all__ = [
    "gaussian_spot",
    "poisson_frame",
    "SinglePair",
    "single_pair",
    "FrameStream",
    "frame_stream",
    "random_texture",
]


def _pixel_integral_1d(n: int, c: float, sigma: float) -> np.ndarray:
    """Integral of exp(-(t-c)^2 / (2 sigma^2)) over each unit pixel [i-1/2, i+1/2]."""
    i = np.arange(n, dtype=np.float64)
    s = math.sqrt(2.0) * sigma
    return sigma * math.sqrt(math.pi / 2.0) * (erf((i + 0.5 - c) / s) - erf((i - 0.5 - c) / s))


def gaussian_spot(H: int, W: int, y0: float, x0: float, sigma: float,
                  amplitude: float, background: float, dark_spot: bool = False) -> np.ndarray:
    """Expected photon counts of a pixel-integrated isotropic Gaussian (Sec. IV).

    ``amplitude`` is the peak of the continuous Gaussian, so the spot holds
    N_gamma = 2 pi sigma^2 amplitude photons. ``background`` is a constant level
    added before noise. ``dark_spot`` subtracts the spot from the background
    instead (the dark particle on a bright background of Sec. IV).
    Returns float64 (H, W).
    """
    gy = _pixel_integral_1d(H, y0, sigma)
    gx = _pixel_integral_1d(W, x0, sigma)
    spot = amplitude * np.outer(gy, gx)
    return background - spot if dark_spot else background + spot


def poisson_frame(rng: np.random.Generator, mu: np.ndarray) -> np.ndarray:
    """One Poisson draw per pixel (shot noise), float64 integers."""
    return rng.poisson(mu).astype(np.float64)


def random_texture(rng: np.random.Generator, H: int, W: int, smooth: float = 1.5) -> np.ndarray:
    """A positive, smooth random texture (non-Gaussian reference for invariance tests)."""
    g = rng.standard_normal((H, W))
    ky = np.fft.fftfreq(H)[:, None]
    kx = np.fft.fftfreq(W)[None, :]
    filt = np.exp(-2.0 * (math.pi * smooth) ** 2 * (ky ** 2 + kx ** 2))
    t = np.real(np.fft.ifft2(np.fft.fft2(g) * filt))
    t = (t - t.min()) / (t.max() - t.min())
    return 50.0 + 1000.0 * t


@dataclass
class SinglePair:
    ref: np.ndarray        # float32 (H, W), noise-free
    frame: np.ndarray      # float32 (H, W), Poisson
    d_true: tuple          # (dx, dy)
    sigma: float
    amplitude: float
    background: float


def single_pair(seed: int = 0, H: int = 64, W: int = 64, sigma: float = 3.0,
                amplitude: float = 1000.0, background: float = 10.0,
                d: tuple = (0.37, -1.21)) -> SinglePair:
    """Single reference/frame pair: FP32, reference centred at (H/2, W/2), frame shifted by d."""
    rng = np.random.default_rng(seed)
    cy, cx = H / 2.0, W / 2.0
    ref = gaussian_spot(H, W, cy, cx, sigma, amplitude, background)
    mu = gaussian_spot(H, W, cy + d[1], cx + d[0], sigma, amplitude, background)
    frame = poisson_frame(rng, mu)
    return SinglePair(ref.astype(np.float32), frame.astype(np.float32), (float(d[0]), float(d[1])),
                      sigma, amplitude, background)


@dataclass
class FrameStream:
    ref: np.ndarray        # float32 (H, W), noise-free
    frames: np.ndarray     # uint16 (n, H, W)
    d_true: np.ndarray     # float64 (n, 2) = (dx, dy) per frame


def brownian_trajectory(rng: np.random.Generator, n: int, step: float, bound: float) -> np.ndarray:
    """d_0 = 0, d_{t+1} = d_t + N(0, step^2) per axis, reflected into [-bound, bound]."""
    d = np.zeros((n, 2))
    steps = rng.normal(0.0, step, size=(n, 2))
    cur = np.zeros(2)
    for t in range(n):
        d[t] = cur
        cur = cur + steps[t]
        for a in range(2):
            while cur[a] > bound or cur[a] < -bound:
                cur[a] = 2 * bound - cur[a] if cur[a] > bound else -2 * bound - cur[a]
    return d


def frame_stream(seed: int = 0, n: int = 10_000, H: int = 128, W: int = 128, sigma: float = 2.5,
                 amplitude: float = 2000.0, background: float = 20.0, step: float = 0.3,
                 bound: float = 24.0, start: int = 0, count: int | None = None) -> FrameStream:
    """Stream of uint16 frames of a spot on a reflected 2-D Brownian trajectory.

    The reference is the noise-free spot at (H/2, W/2). ``start``/``count``
    return a slice of the stream while keeping the draws identical to the full
    stream (noise is drawn frame by frame in order, so earlier frames' draws are
    consumed and discarded).
    """
    rng = np.random.default_rng(seed)
    cy, cx = H / 2.0, W / 2.0
    ref = gaussian_spot(H, W, cy, cx, sigma, amplitude, background)
    d = brownian_trajectory(rng, n, step, bound)
    if count is None:
        count = n - start
    frames = np.empty((count, H, W), dtype=np.uint16)
    for t in range(start + count):
        mu = gaussian_spot(H, W, cy + d[t, 1], cx + d[t, 0], sigma, amplitude, background)
        f = rng.poisson(mu)
        if t >= start:
            frames[t - start] = np.minimum(f, 65535).astype(np.uint16)
    return FrameStream(ref.astype(np.float32), frames, d[start:start + count].copy())


@dataclass
class AdjointPairs:
    ref: np.ndarray        # float32 (H, W), noise-free spot at the centre
    frames: np.ndarray     # float32 (n, H, W), Poisson
    mu: np.ndarray         # float32 (n, H, W), the frames' expected values
    d_true: np.ndarray     # float64 (n, 2) = (dx, dy) per frame


def adjoint_pairs(seed: int = 0, n: int = 1024, H: int = 64, W: int = 64, sigma: float = 3.0,
                  amplitude: float = 1000.0, background: float = 10.0, spread: float = 2.0) -> AdjointPairs:
    """Gradient workload: one noise-free reference, n Poisson frames of the same spot moved by
    (dx, dy) uniform in [-spread, spread] per axis. Draws: shifts, then noise frame by frame."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(-spread, spread, size=(n, 2))
    cy, cx = H / 2.0, W / 2.0
    ref = gaussian_spot(H, W, cy, cx, sigma, amplitude, background)
    mu = np.array([gaussian_spot(H, W, cy + p[1], cx + p[0], sigma, amplitude, background) for p in d])
    frames = np.array([poisson_frame(rng, m) for m in mu])
    return AdjointPairs(ref.astype(np.float32), frames.astype(np.float32), mu.astype(np.float32), d)


@dataclass
class UnevenRois:
    refs: list             # float32 (N_i, N_i) noise-free, one per ROI
    frames: list           # float32 (N_i, N_i), Poisson
    d_true: np.ndarray     # float64 (n, 2) = (dx, dy)


def uneven_rois(seed: int = 0, n: int = 4096, sides=(32, 64, 128)) -> UnevenRois:
    """ROIs of mixed square sizes, each with its own noise-free reference: side uniform over
    `sides`, sigma ~ U(1.5, 4), peak ~ U(200, 5000), background ~ U(5, 50), shift ~ U(-3, 3)^2.
    Draws, per ROI: side, sigma, peak, background, shift, then the noise frame."""
    rng = np.random.default_rng(seed)
    refs, frames, d = [], [], np.zeros((n, 2))
    for i in range(n):
        N = int(rng.choice(np.asarray(sides)))
        sigma, amp, bg = rng.uniform(1.5, 4.0), rng.uniform(200.0, 5000.0), rng.uniform(5.0, 50.0)
        dx, dy = rng.uniform(-3.0, 3.0, size=2)
        d[i] = (dx, dy)
        refs.append(gaussian_spot(N, N, N / 2.0, N / 2.0, sigma, amp, bg).astype(np.float32))
        frames.append(poisson_frame(rng, gaussian_spot(N, N, N / 2.0 + dy, N / 2.0 + dx, sigma, amp, bg))
                      .astype(np.float32))
    return UnevenRois(refs, frames, d)


def camera_pool(seed: int, n: int, N: int, sigma: float = 3.0, amplitude: float = 2000.0,
                background: float = 20.0, spread: float = 3.0):
    """One simulated camera: noise-free reference at the centre and n uint16 Poisson frames
    of the spot moved by (dx, dy) uniform in [-spread, spread]. Draws: shifts, then noise."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(-spread, spread, size=(n, 2))
    ref = gaussian_spot(N, N, N / 2.0, N / 2.0, sigma, amplitude, background).astype(np.float32)
    frames = np.array([poisson_frame(rng, gaussian_spot(N, N, N / 2.0 + p[1], N / 2.0 + p[0], sigma, amplitude,
                                                        background)) for p in d]).astype(np.uint16)
    return ref, frames
