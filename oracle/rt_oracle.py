"""FP64 CPU oracle for the real-time analysis of Sec. III B (arXiv 2310.08770).

TEST INFRASTRUCTURE ONLY, like ``cc_oracle``: only the test-suite, the smoke check
and the benchmark's CPU leg may import it; the product path never calls it.

What it computes, in float64:

1. The aligned frame of Eq. (9), F[I_i(r - r0)]. The paper's r0 is -d for the reported
   displacement d (frame(r) ~ ref(r - d)), so this is F[I_i(r + d)] = F[I_i] times
   e^{+2 pi i (ky' dy / H + kx' dx / W)}. The signed frequencies follow the numpy
   ``fftfreq`` order. On an even axis the Nyquist bin takes the real part cos(pi d) of its
   phase, which keeps the aligned frame, and with it the reference, real.
2. The real-time reference, Eq. (9): F[E_0] = F[I_0], and for i >= 1
   F[E_i] = a0 F[I_i(r + d_i)] + b1 F[E_{i-1}], with a0 = 1 - exp(-T/tau) and
   b1 = exp(-T/tau). Frame i is tracked against E_{i-1} (``cc_oracle.track_one``) before E is
   updated with it. Frame 0 defines E_0 and is not tracked.
   For CC-SN the paper substitutes I -> I'^2 and E -> 1/E, and never says how eps
   enters the reference. This oracle filters E' = E + eps on the aligned I' = I + eps
   and forms the operand 1/E' from it: averaging I'^2 instead would give an image in the
   units of I^2, not of E, and E' = E + eps is exactly the offset reference the fixed-
   reference CC-SN uses. So the CC-SN reference passed to ``track_one`` is E' - eps.
   Spectra are taken with ``cc_oracle``'s naive separable DFTs.
3. Drift removal, Eq. (10): R_0 = a0 r_0, R_n = a0 r_n + b1 R_{n-1}; output r_n - R_n.
4. Rate-limited drift removal, Eqs. (11)-(12): dR_n = a0 r_n + (b1 - 1) R_{n-1}. A step
   longer than alpha/u is cut to length alpha/u along dR_n. R_0 follows Eq. (10)'s start,
   R_0 = a0 r_0 (the paper states no other start).

Pins: ``tests/test_rt_oracle_pins.py``.
"""
from __future__ import annotations

import math

import numpy as np

from . import cc_oracle as co


def axis_phase(N: int, d: float) -> np.ndarray:
    """e^{+2 pi i k' d / N} over the fftfreq-ordered signed frequencies k' of an axis of
    length N; an even N's Nyquist bin (k' = -N/2) gets cos(pi d)."""
    k = co.signed_freq(N)
    ph = np.exp(2j * np.pi * k * d / N)
    if N % 2 == 0:
        ph[N // 2] = math.cos(math.pi * d)
    return ph


def shift_spectrum(F: np.ndarray, dy: float, dx: float) -> np.ndarray:
    """F[I(r + d)] from the full H x W spectrum F = F[I] (item 1 above)."""
    H, W = F.shape
    return F * axis_phase(H, dy)[:, None] * axis_phase(W, dx)[None, :]


def rt_track(frames, u: int = 100, a0: float = 0.05, b1: float | None = None, method: int = co.CC_U,
             eps: float = 200.0) -> list:
    """Real-time tracking of Sec. III B over frames (n, H, W): returns track_one results for
    frames 1 .. n-1, each against the reference filtered from the frames before it."""
    frames = np.asarray(frames, dtype=np.float64)
    if b1 is None:
        b1 = 1.0 - a0
    off = eps if method == co.CC_SN else 0.0
    FE = co.dft2(frames[0] + off)                   # F[E_0] = F[I_0] (I'_0 for CC-SN)
    out = []
    for i in range(1, len(frames)):
        E = np.real(co.idft2(FE)) - off
        r = co.track_one(frames[i], E, u, method, eps)
        out.append(r)
        FI = co.dft2(frames[i] + off)
        FE = a0 * shift_spectrum(FI, r["dy"], r["dx"]) + b1 * FE
    return out


def drift_filter(r, a0: float, b1: float) -> np.ndarray:
    """Eq. (10) over displacements r (n, 2): returns the filtered r_n - R_n."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    R = a0 * r[0]
    out[0] = r[0] - R
    for n in range(1, len(r)):
        R = a0 * r[n] + b1 * R
        out[n] = r[n] - R
    return out


def drift_filter_limited(r, a0: float, b1: float, alpha: float, u: int) -> np.ndarray:
    """Eqs. (11)-(12) over displacements r (n, 2): returns r_n - R_n with the offset's step
    limited to alpha / u."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    lim = alpha / u
    R = a0 * r[0]
    out[0] = r[0] - R
    for n in range(1, len(r)):
        dR = a0 * r[n] + (b1 - 1.0) * R
        norm = math.hypot(dR[0], dR[1])
        R = R + (lim / norm) * dR if norm > lim else R + dR
        out[n] = r[n] - R
    return out
