"""Pins of the continuous-peak / adjoint oracle against mathematics: direct sums, finite
differences of its own closed forms, exact shifts, symmetries, invariances and the
Cramer-Rao bound. CPU only."""
import numpy as np
import pytest

from oracle import adjoint_oracle as ad
from oracle import cc_oracle as co
from paper_2310_08770_b300 import synth


def _pair(H=32, W=32, d=(0.37, -1.21), seed=0, sigma=2.5, amp=1000.0, bg=10.0, noise=True):
    ref = synth.gaussian_spot(H, W, H / 2, W / 2, sigma, amp, bg)
    mu = synth.gaussian_spot(H, W, H / 2 + d[0], W / 2 + d[1], sigma, amp, bg)
    frame = np.random.default_rng(seed).poisson(mu).astype(np.float64) if noise else mu
    return frame, ref


def test_interpolant_at_integer_shifts_is_the_direct_sum():
    rng = np.random.default_rng(1)
    a, b = rng.normal(size=(8, 12)), rng.normal(size=(8, 12))
    X = np.fft.fft2(a) * np.conj(np.fft.fft2(b))
    for s in [(0, 0), (1, 3), (-3, 5), (4, -6)]:
        direct = sum(a[(y + s[0]) % 8, (x + s[1]) % 12] * b[y, x] for y in range(8) for x in range(12))
        assert abs(ad.surface_derivatives(X, np.array(s, float))[0] - direct) < 1e-12


def test_derivatives_match_finite_differences_of_the_interpolant():
    rng = np.random.default_rng(2)
    X = np.fft.fft2(rng.normal(size=(16, 10))) * np.conj(np.fft.fft2(rng.normal(size=(16, 10))))
    s, h = np.array([0.31, -1.7]), 1e-5
    f, g, Hs = ad.surface_derivatives(X, s)
    for i in range(2):
        e = np.zeros(2)
        e[i] = h
        fp, gp, _ = ad.surface_derivatives(X, s + e)
        fm, gm, _ = ad.surface_derivatives(X, s - e)
        assert abs((fp - fm) / (2 * h) - g[i]) < 1e-6 * np.abs(g).max()
        assert np.allclose((gp - gm) / (2 * h), Hs[:, i], rtol=0, atol=1e-6 * np.abs(Hs).max())


def test_band_limited_shift_gives_the_exact_continuous_peak():
    # I(r) = E(r - d) for an image with no energy at or near Nyquist: X = |F[E]|^2 e^{-2 pi i k.d},
    # whose interpolant peaks at exactly d (any d, on or off the grid)
    H, W = 32, 24
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)

    def img(dy, dx):
        return (5.0 + np.cos(2 * np.pi * (2 * (y - dy) / H + 3 * (x - dx) / W))
                + 0.6 * np.sin(2 * np.pi * (-1 * (y - dy) / H + 2 * (x - dx) / W)) + 0.3 * np.cos(2 * np.pi * (y - dy) / H))
    d = np.array([0.4137, -1.2291])
    pk = ad.continuous_peak(img(*d), img(0, 0), np.round(d * 100) / 100)
    assert pk["ok"] and np.allclose(pk["s"], d, atol=1e-10)


def test_exact_integer_roll_gives_the_integer_peak():
    # CC-U: X = |F[E]|^2 e^{-2 pi i k.d}, so Re f(s) <= f(d) with equality only at s = d. (CC-SN
    # has no such bound: its interpolant may dip below the integer minimum between samples.)
    method = co.CC_U
    rng = np.random.default_rng(3)
    E = 100 + 50 * synth.random_texture(rng, 24, 24) + synth.gaussian_spot(24, 24, 11.3, 12.8, 2.0, 500.0, 0.0)
    for d in [(0, 0), (2, -3), (-5, 4)]:
        pk = ad.continuous_peak(np.roll(E, d, axis=(0, 1)), E, (d[0] + 0.02, d[1] - 0.03), method)
        assert pk["ok"] and np.allclose(pk["s"], d, atol=1e-11)


def test_swapping_frame_and_reference_flips_the_continuous_peak():
    frame, ref = _pair(d=(0.41, -0.77), seed=4)
    p1 = ad.continuous_peak(frame, ref, (0.41, -0.77))
    p2 = ad.continuous_peak(ref, frame, (-0.41, 0.77))
    assert np.allclose(p1["s"], -p2["s"], atol=1e-12)


@pytest.mark.parametrize("method", [co.CC_U, co.CC_SN])
def test_vjp_matches_central_differences(method):
    frame, ref = _pair(d=(0.37, -1.21), seed=5)
    rec = co.track_one(frame, ref, 100, method)
    g = (0.7, -1.3)                                     # (dL/ddx, dL/ddy)
    pk, gI, gE = ad.peak_and_vjp(frame, ref, rec, g, method)
    assert pk["ok"]
    h = 1e-3

    def L(F, R):
        s = ad.continuous_peak(F, R, (rec["dy"], rec["dx"]), method)["s"]
        return g[0] * s[1] + g[1] * s[0]
    scale_I, scale_E = np.abs(gI).max(), np.abs(gE).max()
    for (y, x) in [(16, 14), (15, 15), (19, 12), (3, 28), (17, 17)]:
        for img, grad, sc in ((frame, gI, scale_I), (ref, gE, scale_E)):
            p, m = img.copy(), img.copy()
            p[y, x] += h
            m[y, x] -= h
            fd = (L(p, ref) - L(m, ref)) / (2 * h) if img is frame else (L(frame, p) - L(frame, m)) / (2 * h)
            assert abs(fd - grad[y, x]) <= 1e-6 * sc


def test_translating_either_image_moves_the_peak_by_the_translation():
    # d/dt s*(I(r + t e)) = -e and d/dt s*(E(r + t e)) = +e: the VJP dotted with the spectral
    # derivative of the image must give -g (frame) and +g (reference). Exact for CC-U when the
    # images carry no Nyquist energy (a sigma = 3 spot: below 1e-13 there).
    frame, ref = _pair(H=48, W=40, d=(0.23, 0.61), seed=6, sigma=3.0)
    rec = co.track_one(frame, ref, 100)
    H, W = frame.shape
    ky = co.signed_freq(H)[:, None] / H
    kx = co.signed_freq(W)[None, :] / W

    def dimg(img, k):
        return np.real(np.fft.ifft2(np.fft.fft2(img) * 2j * np.pi * k))
    for g in [(1.0, 0.0), (0.0, 1.0), (0.3, -0.8)]:
        _, gI, gE = ad.peak_and_vjp(frame, ref, rec, g)
        gy, gx = g[1], g[0]
        assert abs(np.sum(gI * dimg(frame, ky)) + gy) < 1e-8 and abs(np.sum(gI * dimg(frame, kx)) + gx) < 1e-8
        assert abs(np.sum(gE * dimg(ref, ky)) - gy) < 1e-8 and abs(np.sum(gE * dimg(ref, kx)) - gx) < 1e-8


def test_scaling_an_image_does_not_move_the_peak():
    # CC-U: s* is unchanged by I -> cI and E -> cE (Euler: sum gI I = sum gE E = 0);
    # CC-SN: by E + eps -> c (E + eps) (sum gE (E + eps) = 0)
    frame, ref = _pair(d=(-0.52, 0.18), seed=7)
    for method in (co.CC_U, co.CC_SN):
        rec = co.track_one(frame, ref, 100, method)
        _, gI, gE = ad.peak_and_vjp(frame, ref, rec, (0.9, 0.4), method)
        if method == co.CC_U:
            assert abs(np.sum(gI * frame)) < 1e-10 and abs(np.sum(gE * ref)) < 1e-10
        else:
            assert abs(np.sum(gE * (ref + 200.0))) < 1e-10


def test_propagated_poisson_variance_is_above_the_cramer_rao_bound():
    # the linearised estimator's variance sum_r (ds*/dI(r))^2 mu(r) cannot beat the bound of
    # an unbiased estimator (config: 64 x 64, sigma 3, peak 1000, background 10)
    H = W = 64
    d = (0.37, -1.21)
    ref = synth.gaussian_spot(H, W, 32, 32, 3.0, 1000.0, 10.0)
    mu = synth.gaussian_spot(H, W, 32 + d[0], 32 + d[1], 3.0, 1000.0, 10.0)
    h = 1e-4
    dmu_dy = (synth.gaussian_spot(H, W, 32 + d[0] + h, 32 + d[1], 3.0, 1000.0, 10.0)
              - synth.gaussian_spot(H, W, 32 + d[0] - h, 32 + d[1], 3.0, 1000.0, 10.0)) / (2 * h)
    dmu_dx = (synth.gaussian_spot(H, W, 32 + d[0], 32 + d[1] + h, 3.0, 1000.0, 10.0)
              - synth.gaussian_spot(H, W, 32 + d[0], 32 + d[1] - h, 3.0, 1000.0, 10.0)) / (2 * h)
    bound = ad.crlb(mu, dmu_dy, dmu_dx)
    for method in (co.CC_U, co.CC_SN):
        pk = ad.continuous_peak(mu, ref, d, method)
        sd = []
        for g in [(0.0, 1.0), (1.0, 0.0)]:                 # dL/ds* = e_y, then e_x
            gI, _ = ad.vjp(mu, ref, pk["s"], pk["hess"], g, method)
            sd.append(np.sqrt(np.sum(gI ** 2 * mu)))
        assert np.all(np.array(sd) >= bound * (1 - 1e-9))
        assert np.all(np.array(sd) <= 3.0 * bound)
