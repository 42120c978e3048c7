"""Pins of the offline oracle (Sec. III A, Eq. (8)) against mathematics and the
fixed-reference oracle. CPU only."""
import numpy as np
import pytest

from oracle import cc_oracle as co
from oracle import offline_oracle as off
from paper_2310_08770_b300 import synth


def _texture_spot(H, W, seed):
    rng = np.random.default_rng(seed)
    return synth.gaussian_spot(H, W, H / 2 - 0.7, W / 2 + 0.6, 2.5, 900.0, 15.0) + 50 * synth.random_texture(rng, H, W)


def test_aligned_mean_of_scaled_integer_rolls():
    # frame i = c_i S(r - d_i): moved back by d_i every frame is c_i S, the mean is mean(c) S
    S = _texture_spot(16, 24, 0)
    ds = [(0, 0), (3, -5), (-7, 11), (8, 2)]
    c = np.array([1.0, 0.5, 2.0, 1.3])
    frames = [ci * np.roll(S, d, axis=(0, 1)) for ci, d in zip(c, ds)]
    F = off.aligned_mean(frames, ds)
    assert np.allclose(F, c.mean() * np.fft.fft2(S), rtol=0, atol=1e-9 * np.abs(np.fft.fft2(S)).max())


def test_aligned_mean_of_subpixel_moves_of_a_band_limited_image():
    # a sum of waves below Nyquist moves exactly under the phase ramp: the mean is S itself
    H, W = 32, 24
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)

    def S(dy, dx):
        return (3.0 + np.cos(2 * np.pi * (2 * (y - dy) / H + 3 * (x - dx) / W))
                + 0.4 * np.sin(2 * np.pi * (-5 * (y - dy) / H + 1 * (x - dx) / W)))
    ds = [(0.0, 0.0), (0.37, -1.21), (-2.5, 0.73), (4.01, 3.99)]
    F = off.aligned_mean([S(*d) for d in ds], ds)
    assert np.allclose(np.fft.ifft2(F).real, S(0, 0), atol=1e-12)
    assert np.abs(np.fft.ifft2(F).imag).max() < 1e-12


def test_offset_survives_alignment_as_the_same_constant():
    # the offset of CC-SN is a constant: its spectrum is a DC spike that no phase ramp moves
    rng = np.random.default_rng(1)
    frames = rng.normal(size=(5, 16, 16))
    ds = rng.normal(0, 2, size=(5, 2))
    dF = off.aligned_mean(frames, ds, 200.0) - off.aligned_mean(frames, ds, 0.0)
    want = np.zeros((16, 16), complex)
    want[0, 0] = 200.0 * 256
    assert np.allclose(dF, want, atol=1e-9)


def test_zero_passes_is_the_fixed_reference_frame_zero():
    rng = np.random.default_rng(2)
    frames = np.array([rng.poisson(synth.gaussian_spot(32, 32, 16 + p, 16 - p, 2.0, 800.0, 10.0))
                       for p in (0.0, 0.3, -0.8, 1.4)], dtype=np.float64)
    res, refs = off.offline_track(frames, u=20, passes=0)
    want = co.track_batch(frames, frames[0], u=20)
    # E_0 = I_0 (Eq. (8) before any pass): the DFT round trip returns frame 0 up to rounding
    assert len(res) == 1 and np.max(np.abs(refs[0] - frames[0])) <= 1e-12 * np.abs(frames[0]).max()
    for g, w in zip(res[0], want):
        assert (g["ipy"], g["ipx"], g["dx"], g["dy"]) == (w["ipy"], w["ipx"], w["dx"], w["dy"])


@pytest.mark.parametrize("method", [co.CC_U, co.CC_SN])
def test_integer_rolls_make_frame_zero_a_fixed_point(method):
    # exact rolls are found exactly (both methods, this image), so every aligned frame is I_0
    # and E_n = I_0 for all n
    S = _texture_spot(32, 32, 3)
    ds = [(0, 0), (1, -2), (3, 4), (-5, 2), (2, 2)]
    frames = np.array([np.roll(S, d, axis=(0, 1)) for d in ds])
    res, refs = off.offline_track(frames, u=50, passes=2, method=method)
    for n in range(3):
        assert [(r["dy"], r["dx"]) for r in res[n]] == [tuple(map(float, d)) for d in ds]
        assert np.allclose(refs[n], frames[0], rtol=1e-13, atol=0)


def test_scaled_integer_copies_give_the_mean_scale():
    # frame i = c_i S(r - d_i): CC-U finds d_i - d_0 exactly, so E_1 = mean(c) / c_0 * I_0, and
    # a scaled reference does not move any CC-U maximum
    S = _texture_spot(32, 32, 4)
    ds = [(2, 1), (-3, 4), (5, -6), (0, 0), (7, 7)]
    c = np.array([1.0, 0.6, 1.7, 1.1, 0.9])
    frames = np.array([ci * np.roll(S, d, axis=(0, 1)) for ci, d in zip(c, ds)])
    res, refs = off.offline_track(frames, u=40, passes=1)
    rel = [(dy - ds[0][0], dx - ds[0][1]) for dy, dx in ds]
    assert [(r["dy"], r["dx"]) for r in res[0]] == [tuple(map(float, d)) for d in rel]
    assert np.allclose(refs[1], c.mean() / c[0] * frames[0], rtol=1e-12, atol=0)
    assert [(r["dy"], r["dx"]) for r in res[1]] == [(r["dy"], r["dx"]) for r in res[0]]


def test_single_frame_dataset_is_a_fixed_point():
    rng = np.random.default_rng(5)
    frame = rng.poisson(synth.gaussian_spot(16, 16, 8.3, 7.6, 2.0, 500.0, 10.0)).astype(np.float64)
    res, refs = off.offline_track(frame[None], u=30, passes=3)
    assert all((r[0]["dx"], r[0]["dy"]) == (0.0, 0.0) for r in res)
    assert all(np.allclose(E, frame, rtol=1e-13, atol=1e-12) for E in refs)


def test_noisy_passes_converge_on_the_true_path():
    # noisy streams: the mean of the aligned frames carries less noise than frame 0, so the
    # displacements against E_2 sit closer to the true path than those against E_0 = I_0
    # (mean squared error about a common offset, over ten seeded streams)
    mse = np.zeros(2)
    for seed in range(10, 20):
        rng = np.random.default_rng(seed)
        pos = rng.uniform(-2, 2, size=(24, 2))
        pos[0] = 0
        frames = np.array([rng.poisson(synth.gaussian_spot(32, 32, 16 + p[0], 16 + p[1], 2.0, 300.0, 20.0))
                           for p in pos], dtype=np.float64)
        res, _ = off.offline_track(frames, u=50, passes=2)
        for k, recs in enumerate((res[0], res[2])):
            e = np.array([(r["dy"], r["dx"]) for r in recs]) - pos
            e -= e.mean(axis=0)
            mse[k] += np.mean(np.sum(e ** 2, axis=1))
    assert mse[1] < 0.9 * mse[0]
