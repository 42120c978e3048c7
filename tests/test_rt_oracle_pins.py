"""Pins of the real-time oracle (Sec. III B, Eqs. (9)-(12)) against mathematics and the
fixed-reference oracle. CPU only."""
import math

import numpy as np
import pytest

from oracle import cc_oracle as co
from oracle import rt_oracle as rt
from paper_2310_08770_b300 import synth


def test_integer_alignment_is_an_exact_roll():
    # F[I(r + d)] for integer d: the image rolled by -d, exactly (Nyquist bins: cos(pi d) = +-1)
    rng = np.random.default_rng(0)
    I = rng.normal(size=(16, 12))
    for dy, dx in [(0, 0), (1, 0), (0, -3), (5, 7), (-8, 6)]:
        J = np.fft.ifft2(rt.shift_spectrum(np.fft.fft2(I), dy, dx))
        assert np.max(np.abs(J.imag)) < 1e-12
        assert np.allclose(J.real, np.roll(I, (-dy, -dx), axis=(0, 1)), atol=1e-12)


def test_subpixel_alignment_of_a_band_limited_wave_is_exact():
    H, W = 32, 24
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    dy, dx = 0.37, -1.21
    I = np.cos(2 * np.pi * (3 * y / H + 5 * x / W)) + 0.5 * np.sin(2 * np.pi * (-2 * y / H + 1 * x / W))
    want = (np.cos(2 * np.pi * (3 * (y + dy) / H + 5 * (x + dx) / W))
            + 0.5 * np.sin(2 * np.pi * (-2 * (y + dy) / H + 1 * (x + dx) / W)))
    J = np.fft.ifft2(rt.shift_spectrum(np.fft.fft2(I), dy, dx))
    assert np.allclose(J.real, want, atol=1e-12) and np.max(np.abs(J.imag)) < 1e-12


def test_subpixel_alignment_keeps_real_images_real():
    # the Nyquist rows/columns take cos(pi d): the aligned image of a real frame is real
    rng = np.random.default_rng(1)
    I = rng.normal(size=(16, 16))
    J = np.fft.ifft2(rt.shift_spectrum(np.fft.fft2(I), 0.31, -0.77))
    assert np.max(np.abs(J.imag)) < 1e-12


def _spot_stream(n, H=32, W=32, step=0.4, seed=0, integer=False, noise=True):
    rng = np.random.default_rng(seed)
    pos = np.cumsum(rng.normal(0, step, size=(n, 2)), axis=0)
    pos -= pos[0]
    if integer:
        pos = np.round(pos)
    frames = []
    for p in pos:
        mu = synth.gaussian_spot(H, W, H / 2 + p[0], W / 2 + p[1], 2.0, 800.0, 10.0)
        frames.append(rng.poisson(mu).astype(np.float64) if noise else mu)
    return np.array(frames), pos


@pytest.mark.parametrize("method", [co.CC_U, co.CC_SN])
def test_frozen_filter_equals_fixed_reference(method):
    # a0 = 0, b1 = 1: E_i = E_0 = I_0 for all i, i.e. the fixed-reference path with ref = frame 0
    frames, _ = _spot_stream(6, seed=2)
    got = rt.rt_track(frames, u=20, a0=0.0, b1=1.0, method=method)
    want = co.track_batch(frames[1:], frames[0], u=20, method=method)
    for g, w in zip(got, want):
        assert (g["ipy"], g["ipx"], g["dx"], g["dy"]) == (w["ipy"], w["ipx"], w["dx"], w["dy"])


def test_memoryless_filter_on_integer_moves_realigns_to_frame_zero():
    # a0 = 1, b1 = 0: E_i = I_i(r + d_i). Noise-free frames moved by whole pixels are
    # rolled back onto frame 0 exactly, so every frame is tracked as against frame 0
    frames, pos = _spot_stream(7, seed=3, integer=True, noise=False)
    got = rt.rt_track(frames, u=10, a0=1.0, b1=0.0)
    want = co.track_batch(frames[1:], frames[0], u=10)
    for g, w, p in zip(got, want, pos[1:]):
        assert (g["dx"], g["dy"]) == (w["dx"], w["dy"]) == (p[1], p[0])


def test_low_pass_reference_follows_the_spot():
    # a moving spot tracked with a slowly filtered reference: the reference stays aligned
    # with frame 0, so the displacements follow the true path
    frames, pos = _spot_stream(20, seed=4, step=0.3)
    got = rt.rt_track(frames, u=50, a0=0.2)
    err = [math.hypot(g["dx"] - p[1], g["dy"] - p[0]) for g, p in zip(got, pos[1:])]
    assert max(err) < 0.15


def test_drift_filter_closed_form_for_a_constant_offset():
    a0, c = 0.1, np.array([0.3, -1.2])
    b1 = 1 - a0
    r = np.tile(c, (50, 1))
    out = rt.drift_filter(r, a0, b1)
    n = np.arange(50)[:, None]
    assert np.allclose(out, c * b1 ** (n + 1), atol=1e-15)


def test_drift_filter_is_linear_and_removes_slow_drift():
    rng = np.random.default_rng(5)
    a0 = 0.02
    b1 = 1 - a0
    r1, r2 = rng.normal(size=(400, 2)), rng.normal(size=(400, 2))
    assert np.allclose(rt.drift_filter(2 * r1 - r2, a0, b1),
                       2 * rt.drift_filter(r1, a0, b1) - rt.drift_filter(r2, a0, b1), atol=1e-12)
    ramp = np.linspace(0, 4, 4000)[:, None] * np.array([1.0, 0.5])
    out = rt.drift_filter(ramp, 0.05, 0.95)
    # a ramp of slope s leaves a steady lag of s * b1 / a0 behind the low-pass
    s = np.array([1.0, 0.5]) * 4 / 3999
    assert np.allclose(out[-1], s * 0.95 / 0.05, rtol=1e-6)


def test_limited_drift_equals_eq10_when_steps_are_small():
    rng = np.random.default_rng(6)
    r = rng.normal(0, 0.01, size=(300, 2))
    a0 = 0.05
    assert np.allclose(rt.drift_filter_limited(r, a0, 1 - a0, alpha=0.5, u=1),
                       rt.drift_filter(r, a0, 1 - a0), atol=1e-15)


def test_limited_drift_moves_alpha_over_u_per_frame():
    # a large constant offset: every step is cut to alpha/u along the offset's direction
    c = np.array([3.0, 4.0])
    r = np.tile(c, (30, 1))
    a0, alpha, u = 0.1, 0.5, 100
    out = rt.drift_filter_limited(r, a0, 1 - a0, alpha, u)
    R = c - out
    steps = np.linalg.norm(np.diff(R, axis=0), axis=1)
    assert np.allclose(steps, alpha / u, atol=1e-15)
    d = R[1:] - R[0]
    assert np.allclose(R[0], a0 * c) and np.allclose(d[:, 0] * c[1] - d[:, 1] * c[0], 0.0, atol=1e-12)
