"""Pins of the template-refinement oracle (``oracle.refine_oracle``).

Each check compares it with something it does not compute itself: central finite
differences of its own loss (the gradient), a first-order Taylor prediction (the descent
step), an exact fixed point (targets equal to the peaks), and the halving rule on a step
that must overshoot.
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint_oracle as ad
from oracle import refine_oracle as rf
from paper_2310_08770_b300 import synth


def workload(n=12, H=32, W=32, seed=0, sigma=2.5, amp=800.0, bg=10.0):
    """A noisy template (one Poisson frame at the centre) and calibration frames at known
    uniform shifts, as in the benchmark's refinement leg but smaller."""
    rng = np.random.default_rng(seed)
    E0 = rng.poisson(synth.gaussian_spot(H, W, H / 2, W / 2, sigma, amp, bg)).astype(float)
    d = rng.uniform(-1.5, 1.5, size=(n, 2))
    frames = np.array([rng.poisson(synth.gaussian_spot(H, W, H / 2 + p[1], W / 2 + p[0], sigma, amp, bg))
                       for p in d], float)
    return frames, E0, d


@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_gradient_matches_central_differences(method):
    frames, E0, d = workload(n=6)
    L0, G = rf.loss_and_grad(frames, E0, d, u=50, method=method)
    rng = np.random.default_rng(3)
    h = 1e-3
    for r in [(16, 16), (15, 18), (10, 20)] + [tuple(x) for x in rng.integers(0, 32, size=(3, 2))]:
        Ep, Em = E0.copy(), E0.copy()
        Ep[r] += h
        Em[r] -= h
        fd = (rf.loss_and_grad(frames, Ep, d, u=50, method=method)[0] -
              rf.loss_and_grad(frames, Em, d, u=50, method=method)[0]) / (2 * h)
        assert abs(fd - G[r]) <= 1e-4 * np.abs(G).max() + 1e-12, (r, fd, G[r])


def test_first_step_follows_the_first_order_prediction():
    frames, E0, d = workload(n=8, seed=1)
    L0, G = rf.loss_and_grad(frames, E0, d, u=50)
    h = 1e-4
    step = h * np.linalg.norm(E0) / np.linalg.norm(G)
    L1, _ = rf.loss_and_grad(frames, E0 - step * G, d, u=50)
    predicted = step * np.sum(G * G)                 # first-order decrease
    assert L1 < L0
    assert abs((L0 - L1) - predicted) <= 0.1 * predicted


def test_exact_targets_are_a_fixed_point():
    # targets equal to the continuous peaks at E0: zero loss, zero gradient, E unchanged
    frames, E0, _ = workload(n=5, seed=2)
    peaks = []
    for f in frames:
        r = oracle.track_one(f, E0, 50)
        pk = ad.continuous_peak(f, E0, (r["dy"], r["dx"]))
        peaks.append((pk["s"][1], pk["s"][0]))
    E, hist = rf.refine(frames, E0, np.array(peaks), steps=2, step_rel=0.01, u=50)
    assert np.all(hist[:, 0] <= 1e-24) and np.array_equal(E, E0)


def test_overshooting_step_is_undone_and_halved():
    frames, E0, d = workload(n=8, seed=4)
    E, hist = rf.refine(frames, E0, d, steps=3, step_rel=0.8, u=50)
    # a step of 80% of |E| cannot lower the loss: evaluation 1 is rejected and h halves
    assert hist[1, 0] > hist[0, 0] and hist[1, 1] == 0.8 and hist[2, 1] == 0.4
    accepted = [hist[0, 0]]
    for L, _ in hist[1:]:
        if L <= accepted[-1]:
            accepted.append(L)
    # the returned template is the last accepted one: its loss is the smallest accepted
    L_E, _ = rf.loss_and_grad(frames, E, d, u=50)
    assert abs(L_E - accepted[-1]) <= 1e-15 * max(1.0, accepted[-1])


def test_small_steps_lower_the_loss_monotonically():
    frames, E0, d = workload(n=10, seed=5)
    _, hist = rf.refine(frames, E0, d, steps=4, step_rel=0.002, u=50)
    assert np.all(np.diff(hist[:, 0]) < 0), hist
