"""FP64 CPU oracle for the continuous peak and its adjoint (vector-Jacobian product).

TEST INFRASTRUCTURE ONLY, like ``cc_oracle``: only the test-suite, the smoke check
and the benchmark's CPU leg may import it; the product path never calls it.

The paper's estimate is the extremum of the cross-correlation on the 1/u grid of Sec. III,
a piecewise-constant function of the pixels. What is differentiated here is the extremum
of the same band-limited interpolant without the grid, the u -> infinity limit:

  f(s) = (1/HW) Re sum_k X(k) e^{2 pi i (ky' sy / H + kx' sx / W)},  X = F[a] conj F[b],

over all H x W frequencies with fftfreq-signed ky', kx' (the interpolant the grid samples,
Sec. III; the surface of Eqs. (4) / (7)). (a, b) = (I, E) for CC-U and ((I + eps)^2,
1 / (E + eps)) for CC-SN. s* is the stationary point of f reached by Newton's method from
the grid peak (the tracker's record): a maximum for CC-U, a minimum for CC-SN.

The adjoint follows from grad f(s*) = 0 (implicit function theorem). With Hf the 2 x 2
Hessian of f at s* and an upstream gradient g = dL/ds*, w = -Hf^{-1} g, and for any input
theta: dL/dtheta = w . d(grad_s f)/dtheta. With a and b:

  dL/da(r) = (1/HW) Re sum_k (2 pi i w.k'/N) conj F[b](k) e^{2 pi i k.(s* - r)/N}
  dL/db(r) = (1/HW) Re sum_k (2 pi i w.k'/N) F[a](k) e^{2 pi i k.(s* + r)/N}

(w.k'/N = w_y ky'/H + w_x kx'/W), then the chain rule to pixels: CC-U dL/dI = dL/da,
dL/dE = dL/db; CC-SN dL/dI = 2 (I + eps) dL/da, dL/dE = -dL/db / (E + eps)^2.
The sums over k use ``cc_oracle``'s naive separable DFTs (plain matrix products).

Coordinates are (y, x) throughout; records carry (dy, dx).
Pins: ``tests/test_adjoint_oracle_pins.py``.
"""
from __future__ import annotations

import numpy as np

from . import cc_oracle as co


def operands(frame, ref, method: int = co.CC_U, eps: float = 200.0):
    I = np.asarray(frame, dtype=np.float64)
    E = np.asarray(ref, dtype=np.float64)
    if method == co.CC_SN:
        return (I + eps) ** 2, 1.0 / (E + eps)
    return I, E


def _freqs(H, W):
    ky = co.signed_freq(H)[:, None] / H
    kx = co.signed_freq(W)[None, :] / W
    return ky, kx


def surface_derivatives(X, s):
    """f, grad f (y, x) and the Hessian [[fyy, fyx], [fxy, fxx]] of the interpolant at s."""
    H, W = X.shape
    ky, kx = _freqs(H, W)
    ph = X * np.exp(2j * np.pi * (ky * s[0] + kx * s[1])) / (H * W)
    ty, tx = 2j * np.pi * ky, 2j * np.pi * kx
    f = np.sum(ph).real
    grad = np.array([np.sum(ty * ph).real, np.sum(tx * ph).real])
    hyy = np.sum(ty * ty * ph).real
    hxy = np.sum(ty * tx * ph).real
    hxx = np.sum(tx * tx * ph).real
    return f, grad, np.array([[hyy, hxy], [hxy, hxx]])


def continuous_peak(frame, ref, s0, method: int = co.CC_U, eps: float = 200.0, tol: float = 1e-13,
                    max_iter: int = 50) -> dict:
    """Newton's method on grad f = 0 from s0 = (sy, sx), the grid peak.

    Returns s (y, x), the Hessian there, the number of steps and whether it converged
    (step below tol) to an extremum of the method's kind within 1 px of s0."""
    a, b = operands(frame, ref, method, eps)
    X = co.dft2(a) * np.conj(co.dft2(b))
    s = np.array(s0, dtype=np.float64)
    ok, it = False, 0
    for it in range(1, max_iter + 1):
        _, g, Hs = surface_derivatives(X, s)
        step = np.linalg.solve(Hs, g)
        s = s - step
        if np.max(np.abs(step)) < tol:
            ok = True
            break
    f, g, Hs = surface_derivatives(X, s)
    ev = np.linalg.eigvalsh(Hs)
    kind_ok = bool(np.all(ev < 0)) if method == co.CC_U else bool(np.all(ev > 0))
    near = bool(np.max(np.abs(s - np.asarray(s0))) <= 1.0)
    return {"s": s, "hess": Hs, "f": f, "grad": g, "iters": it, "ok": ok and kind_ok and near}


def vjp(frame, ref, s, hess, g, method: int = co.CC_U, eps: float = 200.0):
    """dL/dI and dL/dE (H x W each) for an upstream gradient g = (dL/dsy, dL/dsx) at the
    continuous peak s with Hessian hess."""
    I = np.asarray(frame, dtype=np.float64)
    E = np.asarray(ref, dtype=np.float64)
    a, b = operands(I, E, method, eps)
    H, W = a.shape
    ky, kx = _freqs(H, W)
    w = -np.linalg.solve(hess, np.asarray(g, dtype=np.float64))
    m = 2j * np.pi * (w[0] * ky + w[1] * kx) * np.exp(2j * np.pi * (ky * s[0] + kx * s[1]))
    Za = m * np.conj(co.dft2(b))
    Zb = m * co.dft2(a)
    dLda = np.real(co.dft2(Za)) / (H * W)          # sum_k Za(k) e^{-2 pi i k.r/N}
    dLdb = np.real(co.idft2(Zb))                   # (1/HW) sum_k Zb(k) e^{+2 pi i k.r/N}
    if method == co.CC_SN:
        return 2.0 * (I + eps) * dLda, -dLdb / (E + eps) ** 2
    return dLda, dLdb


def peak_and_vjp(frame, ref, rec, g, method: int = co.CC_U, eps: float = 200.0):
    """Continuous peak from a tracker record (dy, dx) and the VJP for g = (dL/ddx, dL/ddy),
    the order of the record's fields. Returns (peak dict, dL/dI, dL/dE)."""
    pk = continuous_peak(frame, ref, (rec["dy"], rec["dx"]), method, eps)
    gI, gE = vjp(frame, ref, pk["s"], pk["hess"], (g[1], g[0]), method, eps)
    return pk, gI, gE


def crlb(mu, dmu_dy, dmu_dx):
    """Cramer-Rao bound (std, y and x) of the position for Poisson pixels with mean mu and
    mean derivatives dmu_dy, dmu_dx: the inverse of the Fisher matrix sum (dmu)^2 / mu."""
    J = np.array([[np.sum(dmu_dy * dmu_dy / mu), np.sum(dmu_dy * dmu_dx / mu)],
                  [np.sum(dmu_dx * dmu_dy / mu), np.sum(dmu_dx * dmu_dx / mu)]])
    return np.sqrt(np.diag(np.linalg.inv(J)))
