"""Refinement of the reference template by the adjoint (ccst_refine_reference,
ccst_set_reference_image) through the C ABI, against the FP64 oracle
(``oracle.refine_oracle``), a central finite-difference check of the GPU's dL/dE, and a
torch.autograd loop over the continuous-peak Function.

Bar: the loss history within 1e-6 relative and the same step sizes (the accept/reject
decisions agree), the final template within 1e-6 of its largest value (the GPU's
dL/dE is FP32, 2e-6 relative per step, times the step), and records against the refined
reference that meet the tracker's parity bar with the oracle's.
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint_oracle as ad
from oracle import refine_oracle as rf
from paper_2310_08770_b300 import ccst as C
from paper_2310_08770_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08770_b300 import build
    build.build()
    return _t


def workload(n, H, W, seed, sigma=3.0, amp=1000.0, bg=10.0, spread=2.0, u16=False):
    rng = np.random.default_rng(seed)
    E0 = rng.poisson(synth.gaussian_spot(H, W, H / 2, W / 2, sigma, amp, bg)).astype(np.float32)
    d = rng.uniform(-spread, spread, size=(n, 2))
    frames = np.array([rng.poisson(synth.gaussian_spot(H, W, H / 2 + p[1], W / 2 + p[0], sigma, amp, bg))
                       for p in d])
    frames = frames.astype(np.uint16) if u16 else frames.astype(np.float32)
    return frames, E0, d


def to_device(torch, frames):
    if frames.dtype == np.uint16:
        return torch.from_numpy(frames.view(np.int16)).cuda().view(torch.uint16)
    return torch.from_numpy(frames).cuda()


def gpu_refine(torch, frames, E0, d, u, method, steps, step_rel, max_batch=256):
    n, H, W = frames.shape
    t = C.Tracker(E0, upsample=u, method=method, in_dtype="u16" if frames.dtype == np.uint16 else "f32",
                  max_batch=max_batch)
    dev = to_device(torch, frames)
    tgt = torch.from_numpy(np.ascontiguousarray(d, dtype=np.float64)).cuda()
    hist = torch.empty((steps + 1, 2), dtype=torch.float64, device="cuda")
    Eout = torch.empty((H, W), dtype=torch.float64, device="cuda")
    C.ccst_refine_reference(t.ctx, dev, n, 0, tgt, steps, step_rel, hist, Eout)
    C.ccst_sync(t.ctx)
    return t, dev, hist.cpu().numpy(), Eout.cpu().numpy()


@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_refinement_matches_oracle_64x64(torch, method):
    frames, E0, d = workload(24, 64, 64, seed=1)
    t, dev, hist, E = gpu_refine(torch, frames, E0, d, 100, method, steps=4, step_rel=0.01)
    E_o, hist_o = rf.refine(frames.astype(np.float64), E0.astype(np.float64), d, 4, 0.01, 100, method)
    assert np.array_equal(hist[:, 1], hist_o[:, 1]), (hist, hist_o)
    assert np.allclose(hist[:, 0], hist_o[:, 0], rtol=1e-6, atol=0), (hist, hist_o)
    assert np.max(np.abs(E - E_o)) <= 1e-6 * np.abs(E_o).max()
    # the context now tracks against the refined template
    rec = t.empty_results(8)
    C.ccst_track(t.ctx, dev[:8], 8, 0, rec)
    C.ccst_sync(t.ctx)
    got = C.decode(rec)
    for i in range(8):
        o = oracle.track_one(frames[i].astype(np.float64), E_o, 100, method)
        assert (int(got["ipy"][i]), int(got["ipx"][i])) == (o["ipy"], o["ipx"])
        assert abs(float(got["dx"][i]) - o["dx32"]) <= 1e-3 and abs(float(got["dy"][i]) - o["dy32"]) <= 1e-3
    t.close()


def test_refinement_non_square_u16_with_rejections(torch):
    # a first step of 0.5 |E| overshoots: the history shows the rejected steps halving
    frames, E0, d = workload(16, 32, 16, seed=2, sigma=2.0, spread=1.2, u16=True)
    t, _, hist, E = gpu_refine(torch, frames, E0, d, 40, oracle.CC_U, steps=5, step_rel=0.5, max_batch=7)
    t.close()
    E_o, hist_o = rf.refine(frames.astype(np.float64), E0.astype(np.float64), d, 5, 0.5, 40)
    assert np.array_equal(hist[:, 1], hist_o[:, 1]) and hist[2, 1] < hist[1, 1], (hist, hist_o)
    assert np.allclose(hist[:, 0], hist_o[:, 0], rtol=1e-6, atol=0)
    assert np.max(np.abs(E - E_o)) <= 1e-6 * np.abs(E_o).max()


def test_reference_gradient_matches_central_differences(torch):
    # dL/dE of the refinement loss from ccst_backward, against central differences (h = 1e-3)
    # of the oracle's loss at sampled pixels of the template
    frames, E0, d = workload(10, 64, 64, seed=3)
    n = len(frames)
    t = C.Tracker(E0, upsample=100, in_dtype="f32")
    dev = to_device(torch, frames)
    rec = t.empty_results(n)
    C.ccst_track(t.ctx, dev, n, 0, rec)
    peak = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    status = torch.empty((n,), dtype=torch.int32, device="cuda")
    C.ccst_peak_continuous(t.ctx, dev, n, 0, rec, peak, status)
    C.ccst_sync(t.ctx)
    assert status.cpu().tolist() == [0] * n
    g = (2.0 * (peak.cpu().numpy() - d) / n).astype(np.float32)
    gE = torch.empty((64, 64), dtype=torch.float32, device="cuda")
    C.ccst_backward(t.ctx, dev, n, 0, rec, torch.from_numpy(g).cuda(), None, gE)
    C.ccst_sync(t.ctx)
    t.close()
    gE = gE.cpu().numpy()
    E64 = E0.astype(np.float64)
    h = 1e-3
    for r in [(32, 32), (30, 35), (36, 29), (20, 44), (45, 20)]:
        Ep, Em = E64.copy(), E64.copy()
        Ep[r] += h
        Em[r] -= h
        fd = (rf.loss_and_grad(frames.astype(np.float64), Ep, d, 100)[0] -
              rf.loss_and_grad(frames.astype(np.float64), Em, d, 100)[0]) / (2 * h)
        assert abs(fd - gE[r]) <= 1e-4 * np.abs(gE).max(), (r, fd, gE[r])


def test_autograd_loop_gives_the_entry_points_template(torch):
    # a user-side loop: the torch.autograd Function gives dL/dE, a normalised step is taken
    # in torch, and ccst_set_reference_image moves the context's reference; with small
    # steps (no rejection) it follows ccst_refine_reference
    from paper_2310_08770_b300.autograd import continuous_peak
    frames, E0, d = workload(12, 64, 64, seed=4)
    n = len(frames)
    steps, h = 2, 0.003
    t_ref, _, hist, E_entry = gpu_refine(torch, frames, E0, d, 100, oracle.CC_U, steps, h)
    t_ref.close()
    assert np.all(hist[:, 1] == h)                    # no step was rejected
    t = C.Tracker(E0, upsample=100, in_dtype="f32")
    fr = torch.from_numpy(frames).cuda()
    tgt = torch.from_numpy(d).cuda()
    E = torch.from_numpy(E0.astype(np.float64)).cuda()
    for k in range(steps):
        C.ccst_set_reference_image(t.ctx, E)
        leaf = torch.zeros((64, 64), dtype=torch.float32, device="cuda", requires_grad=True)
        peak, status = continuous_peak(t, fr, leaf)
        ok = (status == 0).to(torch.float64)
        loss = (((peak - tgt) ** 2).sum(dim=1) * ok).sum() / n
        loss.backward()
        G = leaf.grad.double()
        E = E - h * torch.linalg.norm(E) / torch.linalg.norm(G) * G
    t.close()
    assert np.max(np.abs(E.cpu().numpy() - E_entry)) <= 1e-6 * np.abs(E_entry).max()


def test_refinement_rejects_bad_arguments(torch):
    frames, E0, d = workload(2, 32, 32, seed=5)
    t = C.Tracker(E0, upsample=20, in_dtype="f32")
    dev = to_device(torch, frames)
    tgt = torch.from_numpy(d).cuda()
    hist = torch.empty((4,), dtype=torch.float64, device="cuda")
    for args in [(dev, 0, 0, tgt, 1, 0.01, hist), (dev, 2, 0, None, 1, 0.01, hist), (dev, 2, 0, tgt, -1, 0.01, hist),
                 (dev, 2, 0, tgt, 1, 0.0, hist), (dev, 2, 0, tgt, 1, float("nan"), hist), (dev, 2, 0, tgt, 1, 0.01, None),
                 (dev, 2, 8, tgt, 1, 0.01, hist)]:
        with pytest.raises(C.CcstError) as e:
            C.ccst_refine_reference(t.ctx, *args)
        assert e.value.code == C.E_INVALID
    with pytest.raises(C.CcstError):
        C.ccst_set_reference_image(t.ctx, None)
    t.close()
    g = C.Tracker(np.ones((48, 48), np.float32), upsample=20, in_dtype="f32")     # a general-shape context
    with pytest.raises(C.CcstError) as e:
        C.ccst_refine_reference(g.ctx, torch.zeros((1, 48, 48), device="cuda"), 1, 0, tgt[:1], 1, 0.01, hist)
    assert e.value.code == C.E_UNSUPPORTED
    g.close()
