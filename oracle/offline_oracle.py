"""FP64 CPU oracle for the offline (iterative) analysis of Sec. III A (arXiv 2310.08770).

TEST INFRASTRUCTURE ONLY, like ``cc_oracle``: only the test-suite, the smoke check
and the benchmark's CPU leg may import it; the product path never calls it.

What it computes, in float64:

1. The reference of Eq. (8): the mean, in Fourier space, of all N frames of a dataset,
   each aligned by the displacement d_i it was given against the previous reference:
   F[E_n] = (1/N) sum_i F[I_i(r + d_i)]. The aligned frame is the one of the real-time
   oracle (``rt_oracle.shift_spectrum``): frame(r) ~ ref(r - d), so I_i(r + d_i) moves
   frame i back onto the reference.
2. The iteration: F[E_0] = F[I_0]. Pass n tracks every frame against E_n with
   ``cc_oracle.track_one``; for n < passes, those displacements give E_{n+1} by item 1.
3. CC-SN (Sec. III: I -> I'^2, E -> 1/E): as in the real-time oracle, the mean is taken of
   the aligned I' = I + eps, giving E' = E + eps, and the operand is 1/E'. The reference
   passed to ``track_one`` is therefore E' - eps.

Pins: ``tests/test_offline_oracle_pins.py``.
"""
from __future__ import annotations

import numpy as np

from . import cc_oracle as co
from . import rt_oracle as rt


def aligned_mean(frames, disp, off: float = 0.0) -> np.ndarray:
    """F[E] of Eq. (8): the mean of F[I_i + off] moved by the displacements disp (N, 2) =
    (dy_i, dx_i); the full H x W spectrum."""
    frames = np.asarray(frames, dtype=np.float64)
    acc = np.zeros(frames.shape[1:], dtype=np.complex128)
    for f, (dy, dx) in zip(frames, np.asarray(disp, dtype=np.float64)):
        acc += rt.shift_spectrum(co.dft2(f + off), dy, dx)
    return acc / len(frames)


def offline_track(frames, u: int = 100, passes: int = 5, method: int = co.CC_U, eps: float = 200.0):
    """The iterative method of Sec. III A over frames (N, H, W).

    Returns (results, refs): results[n] holds the ``track_one`` records of every frame
    against E_n, refs[n] the image E_n, for n = 0 .. passes."""
    frames = np.asarray(frames, dtype=np.float64)
    off = eps if method == co.CC_SN else 0.0
    FE = co.dft2(frames[0] + off)
    results, refs = [], []
    for n in range(passes + 1):
        E = np.real(co.idft2(FE)) - off
        recs = co.track_batch(frames, E, u, method, eps)
        results.append(recs)
        refs.append(E)
        if n < passes:
            FE = aligned_mean(frames, [(r["dy"], r["dx"]) for r in recs], off)
    return results, refs
