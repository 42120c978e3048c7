"""FP64 CPU oracle for refining the reference template by the adjoint of the displacement.

TEST INFRASTRUCTURE ONLY, like ``cc_oracle``: only the test-suite, the smoke check and the
benchmark's CPU leg may import it; the product path never calls it.

The paper refines its reference by averaging aligned frames (Eq. (8), Sec. III A) or by
low-pass filtering them (Eq. (9), Sec. III B). This is a different refinement, with no
counterpart in the paper. The template E is fitted to calibration frames whose
displacements d_i are known, by gradient descent on the mean squared error of their
continuous peaks:

  L(E) = (1/n) sum_{i: peak ok} |s*_i(E) - d_i|^2,   dL/ds*_i = 2 (s*_i - d_i) / n,

where s*_i is the stationary point of the correlation interpolant (``adjoint_oracle``),
reached by Newton's method from the tracker's grid peak (``cc_oracle.track_one``), and
dL/dE = sum_i (VJP of s*_i with respect to E) from ``adjoint_oracle.vjp``.

The step rule, in the order it runs (k = 0 .. steps):
  1. evaluate L(E_k) and dL/dE at E_k; record (L(E_k), h);
  2. if an accepted template exists and L(E_k) > its loss: go back to it and its gradient,
     and halve h; otherwise accept E_k;
  3. unless k = steps: E <- E_acc - h |E_acc|_2 / |G_acc|_2 G_acc, where E_acc is the accepted
     template and G_acc its gradient (2-norms over the pixels).
The result is the last accepted template and the (loss, step) history.
Pins: ``tests/test_refine_oracle_pins.py``.
"""
from __future__ import annotations

import numpy as np

from . import adjoint_oracle as ad
from . import cc_oracle as co


def loss_and_grad(frames, E, target, u: int = 100, method: int = co.CC_U, eps: float = 200.0):
    """L(E) and dL/dE (H x W) over calibration frames (n, H, W) with known (dx, dy) targets."""
    frames = np.asarray(frames, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    n = len(frames)
    loss = 0.0
    grad = np.zeros_like(E)
    for i in range(n):
        rec = co.track_one(frames[i], E, u, method, eps)
        pk = ad.continuous_peak(frames[i], E, (rec["dy"], rec["dx"]), method, eps)
        if not pk["ok"]:
            continue
        ex, ey = pk["s"][1] - target[i, 0], pk["s"][0] - target[i, 1]
        loss += (ex * ex + ey * ey) / n
        _, gE = ad.vjp(frames[i], E, pk["s"], pk["hess"], (2.0 * ey / n, 2.0 * ex / n), method, eps)
        grad += gE
    return loss, grad


def refine(frames, E0, target, steps: int, step_rel: float, u: int = 100, method: int = co.CC_U,
           eps: float = 200.0):
    """The refinement above. Returns (E, history) with history a (steps + 1, 2) array of
    (L(E_k), the step h that produced E_k)."""
    E = np.array(E0, dtype=np.float64)
    h = float(step_rel)
    acc_E = acc_G = None
    acc_L = None
    hist = []
    for k in range(steps + 1):
        L, G = loss_and_grad(frames, E, target, u, method, eps)
        hist.append((L, h))
        if acc_L is not None and L > acc_L:
            h *= 0.5
            E = acc_E
        else:
            acc_E, acc_G, acc_L = E, G, L
        if k == steps:
            break
        norm_g = np.linalg.norm(acc_G)
        coef = h * np.linalg.norm(acc_E) / norm_g if norm_g > 0 else 0.0
        E = acc_E - coef * acc_G
    return acc_E, np.array(hist)
