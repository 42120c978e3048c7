"""Plants plausible mistakes in the oracle (on the CPU) and checks that the pins catch each.

Each mutant replaces one oracle function with a subtly wrong version (a dropped
conjugate, a transposed operand, a wrong sign, index or wrap); the pins of
``test_oracle_pins`` must fail for every one of them.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.cc_oracle as co
import tests.test_oracle_pins as pins
from oracle import CC_SN, CC_U


def _run_pins():
    """Run a fixed selection of pins; return how many failed."""
    checks = [
        pins.test_grid_matches_paper_example,
        lambda: pins.test_direct_sum_equals_dft_route((12, 8), CC_U),
        lambda: pins.test_naive_dft_matches_numpy_fft((5, 7)),
        pins.test_naive_dft_closed_forms,
        pins.test_top2_margin_hand_built,
        pins.test_track_one_margins_hand_built,
        lambda: pins.test_surface_is_chi_square_up_to_constants(CC_U),
        lambda: pins.test_surface_is_chi_square_up_to_constants(CC_SN),
        lambda: pins.test_integer_roll_recovered_exactly_ccu(*pins._refs()[1], 7),
        lambda: pins.test_integer_roll_recovered_exactly_ccu(*pins._refs()[2], 100),
        lambda: pins.test_integer_roll_recovered_ccsn(*pins._refs()[0]),
        lambda: pins.test_noise_free_subpixel_is_nearest_grid_point(100, (0.37, -1.21), 3.0, 64),
        lambda: pins.test_noise_free_subpixel_is_nearest_grid_point(37, (0.9, -0.25), 3.0, 64),
        lambda: pins.test_grid_centre_equals_direct_sum(CC_U),
        lambda: pins.test_upsampled_grid_equals_dirichlet_brute_force((6, 10), 5, CC_U),
        lambda: pins.test_upsampled_grid_equals_dirichlet_brute_force((5, 7), 4, CC_SN),
        pins.test_constant_frame_ties_go_to_lowest_index,
    ]
    failed = 0
    for chk in checks:
        try:
            chk()
        except (AssertionError, ValueError, IndexError):
            failed += 1
    return failed


def test_unmutated_oracle_passes_selection():
    assert _run_pins() == 0


def _m_conj_wrong_operand(a, b):
    return np.conj(co.dft2(np.asarray(a, float))) * co.dft2(np.asarray(b, float))


def _m_dft_forward_sign(a):
    a = np.asarray(a)
    H, W = a.shape
    return co.dft_matrix(H, +1) @ (a @ co.dft_matrix(W, +1))


def _m_dft_index_not_reduced(N, sign=-1):
    # the angle index taken as k + n instead of k n
    k = np.arange(N, dtype=np.int64)
    ang = (2.0 * math.pi / N) * np.add.outer(k, k).astype(np.float64)
    return np.cos(ang) + (1j * sign) * np.sin(ang)


def _m_margin_ignores_sense(values, sense):
    v = np.sort(np.asarray(values).ravel())
    return float(v[-1] - v[-2]) if v.size > 1 else math.inf


def _m_margin_distinct_values(values, sense):
    # exact ties merged: a tied surface would report the gap to the next distinct value
    v = np.unique(np.asarray(values).ravel() * sense)
    return float(v[-1] - v[-2]) if v.size > 1 else math.inf


def _m_margin_best_minus_worst(values, sense):
    v = np.sort(np.asarray(values).ravel() * sense)
    return float(v[-1] - v[0]) if v.size > 1 else math.inf


def _m_grid_floor(u):
    return (3 * int(u)) // 2


def _m_freq_split_odd(N):
    # right for even N; for odd N puts the highest positive bin on the negative side
    k = np.arange(N, dtype=np.int64)
    return np.where(k < N // 2, k, k - N)


def _m_kernel_offset(N, p, u):
    M = co.grid_size(u)
    j = np.arange(M, dtype=np.int64) - (M - 1) // 2
    k = co.signed_freq(N)
    m = np.mod(k[None, :] * (p * u + j[:, None]), u * N)
    ang = (2.0 * math.pi / (u * N)) * m
    return np.cos(ang) + 1j * np.sin(ang)


def _m_kernel_sign(N, p, u):
    return np.conj(co.__dict__["_orig_upsample_kernel"](N, p, u))


def _m_upsampled_transposed(X, py, px, u):
    H, W = X.shape
    Ky = co.upsample_kernel(H, py, u)
    Kx = co.upsample_kernel(W, px, u)
    return np.real(Ky @ X @ Kx) / (H * W) if H == W else np.real((Kx @ X.T @ Ky.T).T) / (H * W)


def _m_upsampled_imag(X, py, px, u):
    H, W = X.shape
    return np.abs(co.upsample_kernel(H, py, u) @ X @ co.upsample_kernel(W, px, u).T) / (H * W)


def _m_wrap(p, N):
    return p - N if p >= N // 2 else p


def _m_operands_no_square(frame, ref, method=CC_U, eps=200.0):
    I = np.asarray(frame, float)
    E = np.asarray(ref, float)
    if method == CC_U:
        return I, E, +1
    return I + eps, 1.0 / (E + eps), -1


def _m_operands_ccsn_max(frame, ref, method=CC_U, eps=200.0):
    a, b, s = co.__dict__["_orig_surface_operands"](frame, ref, method, eps)
    return a, b, +1


def _m_extremum_last(values, sense):
    v = np.asarray(values).ravel() * sense
    return int(len(v) - 1 - np.argmax(v[::-1]))


def _m_direct_roll_sign(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    H, W = a.shape
    c = np.empty((H, W))
    for sy in range(H):
        for sx in range(W):
            c[sy, sx] = np.sum(np.roll(a, (sy, sx), axis=(0, 1)) * b)
    return c


MUTANTS = {
    "conj_on_wrong_operand": ("product_spectrum", _m_conj_wrong_operand),
    "dft_forward_sign": ("dft2", _m_dft_forward_sign),
    "dft_index_not_reduced": ("dft_matrix", _m_dft_index_not_reduced),
    "margin_ignores_sense": ("top2_margin", _m_margin_ignores_sense),
    "margin_merges_ties": ("top2_margin", _m_margin_distinct_values),
    "margin_best_minus_worst": ("top2_margin", _m_margin_best_minus_worst),
    "grid_floor_not_ceil": ("grid_size", _m_grid_floor),
    # (moving the Nyquist bin of an even size to +N/2 on both axes is not a mistake:
    #  the real part of the interpolant does not change, so it is not planted here)
    "frequency_split_odd_sizes": ("signed_freq", _m_freq_split_odd),
    "grid_offset_origin": ("upsample_kernel", _m_kernel_offset),
    "kernel_sign": ("upsample_kernel", _m_kernel_sign),
    "transposed_contraction": ("upsampled_cc", _m_upsampled_transposed),
    "modulus_not_real_part": ("upsampled_cc", _m_upsampled_imag),
    "wrap_at_half": ("wrap_shift", _m_wrap),
    "ccsn_without_square": ("surface_operands", _m_operands_no_square),
    "ccsn_maximum": ("surface_operands", _m_operands_ccsn_max),
    "ties_to_last_index": ("extremum_index", _m_extremum_last),
    "direct_sum_shift_sign": ("cc_surface_direct", _m_direct_roll_sign),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, monkeypatch):
    fn_name, mutant = MUTANTS[name]
    monkeypatch.setitem(co.__dict__, "_orig_" + fn_name, getattr(co, fn_name))
    monkeypatch.setattr(co, fn_name, mutant)
    monkeypatch.setattr(oracle, fn_name, mutant)
    assert _run_pins() >= 1, f"no pin caught mutant {name}"
