"""FP64 CPU oracle for cross-correlation sub-pixel tracking (arXiv 2310.08770).

TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check of the package
entry point and the CPU-baseline leg of the benchmark may import or run this
module. The product path (the CUDA library and its Python binding) never calls
it, and it shares no code, table or constant generator with that path.

What it computes, per frame, in float64, as plainly as possible:

1. The surface operands (Sec. II). CC-U: (I, E), Eqs. (2)-(4). CC-SN: (I'^2,
   1/E_SN) with I' = I + eps and E_SN = E + eps, Eqs. (5)-(7).
2. The integer cross-correlation surface c(s) = sum_r a((r+s) mod N) b(r)
   (left-hand side of Eq. (4) / Eq. (7), periodic boundaries as in Eq. (1)),
   by direct summation, or as the right-hand side of Eq. (4) with naive
   separable DFTs: F[a] = D_H a D_W (a row DFT then a column DFT, each a plain
   matrix product with the N x N DFT matrix, no FFT), X = F[a] conj(F[b]), and
   the naive inverse DFT of X. The DFT matrices' angle indices k n are reduced
   mod N exactly in integers. The pin tests check that the two routes agree, and
   check the DFT against numpy's FFT as an independent library.
3. The integer peak: argmax of c for CC-U, argmin for CC-SN (the chi^2
   minimiser of Eq. (6)); ties go to the lowest row-major index; each axis is
   wrapped to (-ceil(N/2), floor(N/2)].
4. The upsampled cross-correlation of Sec. III (the matrix-multiply DFT of its
   ref. [27]): a 1.5-pixel square centred on the integer peak, sampled with
   M = ceil(1.5 u) points per axis at offsets (j - floor(M/2))/u; the product
   spectrum X = F[a] conj(F[b]) is evaluated there by an inverse DFT over all
   H x W frequencies (signed, numpy fftfreq order), real part taken.
   Twiddle angles are reduced exactly in integers.
5. The sub-pixel extremum on that grid (argmax / argmin, lowest row-major
   index on ties) gives d = p + offset; ``peak`` is the surface value there, in
   the units of the direct sum (it equals c(p) at offset 0).

Readings of the paper taken here: the displacement reported is the motion d of
the frame content, frame(r) ~ ref(r - d), i.e. the shift s of the maximum of
c(s) = sum_r I(r+s) E(r) (Eq. (1)'s r0 is -d); CC-SN takes the minimum of
Eq. (7) because that minimises Eq. (6) (the text says maximum, which on a
noise-free shifted spot lands far from the shift); the grid has M = ceil(1.5 u)
points with offsets (j - floor(M/2))/u (the paper's u = 256 gives its 384 x 384);
no windowing or mean subtraction is applied (the paper names none).

Every function below is pinned by tests in ``tests/test_oracle_pins.py``
against values fixed by the paper or by mathematics (exact integer shifts,
sign flip on swapping the images, noise-free sub-pixel Gaussian spots, the
direct-sum vs naive-DFT identity, the naive DFT vs numpy's FFT, the
Dirichlet-kernel brute force on tiny images,
the Poisson Cramer-Rao bound).
"""
from __future__ import annotations

import functools
import math

import numpy as np

CC_U = 0
CC_SN = 1


def grid_size(u: int) -> int:
    """M = ceil(1.5 u): samples per axis of the 1.5-pixel refinement square (Sec. III).

    The paper's example u = 256 gives 384 x 384.
    """
    return (3 * int(u) + 1) // 2


def signed_freq(N: int) -> np.ndarray:
    """Signed DFT frequency of each bin k = 0..N-1: k for k < ceil(N/2), else k - N (int64)."""
    k = np.arange(N, dtype=np.int64)
    return np.where(k < (N + 1) // 2, k, k - N)


def surface_operands(frame, ref, method: int = CC_U, eps: float = 200.0):
    """Operands (a, b) of the correlation surface and the extremum sense.

    CC-U (Sec. II, Eq. (3)-(4)): a = I, b = E, maximum.
    CC-SN (Sec. II, Eq. (5)-(7)): a = (I + eps)^2, b = 1/(E + eps), minimum, because
    Eq. (6) is minimised where sum_r I'(r - r0)^2 / E(r) is smallest.
    Returns (a, b, sense) with sense = +1 for a maximum and -1 for a minimum.
    """
    I = np.asarray(frame, dtype=np.float64)
    E = np.asarray(ref, dtype=np.float64)
    if method == CC_U:
        return I, E, +1
    if method == CC_SN:
        Ip = I + eps
        return Ip * Ip, 1.0 / (E + eps), -1
    raise ValueError("method must be CC_U (0) or CC_SN (1)")


def cc_surface_direct(a, b) -> np.ndarray:
    """c(s) = sum_r a((r + s) mod N) b(r) for every integer shift s, by direct summation.

    Left-hand side of Eq. (4) (and of Eq. (7) with the CC-SN operands), periodic
    boundaries as assumed for Eq. (1). O(H^2 W^2): meant for small images.
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    H, W = a.shape
    c = np.empty((H, W), dtype=np.float64)
    for sy in range(H):
        ay = np.roll(a, -sy, axis=0)          # ay[r] = a[r + sy]
        for sx in range(W):
            c[sy, sx] = np.sum(np.roll(ay, -sx, axis=1) * b)
    return c


@functools.lru_cache(maxsize=64)
def dft_matrix(N: int, sign: int = -1) -> np.ndarray:
    """D[k, n] = exp(sign 2 pi i k n / N), k, n = 0..N-1 (complex128, symmetric).

    The angle index k n is reduced mod N exactly in integers before the trigonometric
    call, so every entry is cos/sin of 2 pi m / N with 0 <= m < N."""
    k = np.arange(N, dtype=np.int64)
    m = np.mod(np.outer(k, k), N)
    ang = (2.0 * math.pi / N) * m.astype(np.float64)
    D = np.cos(ang) + (1j * sign) * np.sin(ang)
    D.setflags(write=False)
    return D


def dft2(a) -> np.ndarray:
    """F[a](k) = sum_n a(n) e^{-2 pi i (ky ny / H + kx nx / W)}: the naive separable DFT,
    a row DFT (a D_W) then a column DFT (D_H (.)), each a plain matrix product."""
    a = np.asarray(a)
    H, W = a.shape
    return dft_matrix(H, -1) @ (a @ dft_matrix(W, -1))


def idft2(X) -> np.ndarray:
    """F^-1[X](n) = (1/HW) sum_k X(k) e^{+2 pi i (ky ny / H + kx nx / W)}, naive and separable."""
    X = np.asarray(X)
    H, W = X.shape
    return (dft_matrix(H, +1) @ (X @ dft_matrix(W, +1))) / (H * W)


def product_spectrum(a, b) -> np.ndarray:
    """X = F[a] (x) conj(F[b]): the element-wise product of Eq. (4) / Eq. (7), complex128,
    with naive DFTs."""
    return dft2(np.asarray(a, np.float64)) * np.conj(dft2(np.asarray(b, np.float64)))


def cc_surface_dft(a, b) -> np.ndarray:
    """c = F^-1[F[a] (x) conj(F[b])]: right-hand side of Eq. (4), with naive DFTs."""
    return np.real(idft2(product_spectrum(a, b)))


def wrap_shift(p: int, N: int) -> int:
    """Map a cyclic shift 0..N-1 to (-ceil(N/2), floor(N/2)]."""
    return p - N if p > N // 2 else p


def extremum_index(values: np.ndarray, sense: int) -> int:
    """Flat index of the maximum (sense=+1) or minimum (sense=-1); lowest index on ties."""
    v = np.asarray(values).ravel()
    return int(np.argmax(v) if sense > 0 else np.argmin(v))


def top2_margin(values: np.ndarray, sense: int) -> float:
    """best - second best of a surface in the extremum's sense (sense=+1: largest minus the
    next largest value; sense=-1: next smallest minus smallest). Repeated values count
    separately, so an exact tie gives 0; a one-element surface gives inf."""
    v = np.sort(np.asarray(values).ravel() * sense)
    return float(v[-1] - v[-2]) if v.size > 1 else math.inf


def upsample_kernel(N: int, p: int, u: int) -> np.ndarray:
    """K[j, k] = exp(+2 pi i k' (p + (j - floor(M/2))/u) / N) for the M grid rows and N bins.

    The angle is 2 pi m / (u N) with m = k' (p u + j - floor(M/2)) reduced mod u N
    exactly in integers before the trigonometric call.
    """
    M = grid_size(u)
    j = np.arange(M, dtype=np.int64) - M // 2
    k = signed_freq(N)
    m = np.mod(k[None, :] * (p * u + j[:, None]), u * N)
    ang = (2.0 * math.pi / (u * N)) * m.astype(np.float64)
    return np.cos(ang) + 1j * np.sin(ang)


def upsampled_cc(X: np.ndarray, py: int, px: int, u: int) -> np.ndarray:
    """Upsampled cross-correlation on the M x M grid around the integer peak (Sec. III).

    cu[jy, jx] = (1/HW) Re sum_{ky,kx} X[ky,kx] exp(2 pi i [ky'(py + oy)/H + kx'(px + ox)/W])
    with o = (j - floor(M/2))/u, evaluated as Ky @ X @ Kx^T (the matrix-multiply
    DFT of the refinement method the paper follows). Row index = y.
    """
    H, W = X.shape
    Ky = upsample_kernel(H, py, u)
    Kx = upsample_kernel(W, px, u)
    return np.real(Ky @ X @ Kx.T) / (H * W)


def track_one(frame, ref, u: int = 100, method: int = CC_U, eps: float = 200.0,
              integer_route: str = "dft") -> dict:
    """Displacement of one frame against the reference (Sec. II-III), all in float64.

    Returns a dict with dx, dy (float64 and their float32 roundings), peak, the
    integer peak (ipy, ipx, wrapped), the flat sub-pixel index j, and the
    relative top-2 margins of the integer and sub-pixel searches (margin divided
    by sum|X|/HW, an upper bound of |c|) that tests use to recognise genuine ties.
    """
    a, b, sense = surface_operands(frame, ref, method, eps)
    H, W = a.shape
    X = product_spectrum(a, b)
    if integer_route == "direct":
        c = cc_surface_direct(a, b)
    elif integer_route == "dft":
        c = np.real(idft2(X))
    else:
        raise ValueError("integer_route must be 'dft' or 'direct'")
    p = extremum_index(c, sense)
    py, px = wrap_shift(p // W, H), wrap_shift(p % W, W)
    cu = upsampled_cc(X, py, px, u)
    M = grid_size(u)
    j = extremum_index(cu, sense)
    jy, jx = divmod(j, M)
    dy = (py * u + jy - M // 2) / u
    dx = (px * u + jx - M // 2) / u
    scale = float(np.sum(np.abs(X))) / (H * W)
    return {
        "dx": dx, "dy": dy,
        "dx32": float(np.float32(dx)), "dy32": float(np.float32(dy)),
        "peak": float(cu[jy, jx]),
        "ipy": py, "ipx": px, "jy": jy, "jx": jx,
        "int_margin": top2_margin(c, sense) / scale if scale > 0 else 0.0,
        "sub_margin": top2_margin(cu, sense) / scale if scale > 0 else 0.0,
        "scale": scale,
    }


def track_batch(frames, ref, u: int = 100, method: int = CC_U, eps: float = 200.0) -> list:
    """track_one over a stack of frames (n, H, W), in order."""
    return [track_one(f, ref, u, method, eps) for f in np.asarray(frames)]


def _worker(args):
    frames, ref, u, method, eps = args
    return track_batch(frames, ref, u, method, eps)


def track_batch_parallel(frames, ref, u: int = 100, method: int = CC_U, eps: float = 200.0,
                         processes: int | None = None) -> list:
    """track_batch split over a 'spawn' process pool (one BLAS thread per worker).

    Used for the timed CPU baseline and for large parity samples; results are
    identical to track_batch.
    """
    import multiprocessing as mp
    import os
    frames = np.asarray(frames)
    n = len(frames)
    procs = processes or os.cpu_count() or 1
    procs = max(1, min(procs, n))
    chunks = np.array_split(np.arange(n), procs)
    ctx = mp.get_context("spawn")
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        with ctx.Pool(procs) as pool:
            parts = pool.map(_worker, [(frames[c], ref, u, method, eps) for c in chunks if len(c)])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    out = []
    for p in parts:
        out.extend(p)
    return out
