"""Continuous peak and its adjoint (ccst_peak_continuous / ccst_backward) through the C ABI,
against the FP64 oracle (``oracle.adjoint_oracle``).

Bar: s* within 1e-9 px of the oracle (both are Newton solutions of the same equation: the
oracle's sums in FP64, the kernel's row sums in double-float, about 2^-46 a term), and the
gradients, returned as float32, within 2e-6 of the largest oracle value of the same image.
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint_oracle as ad
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


def pairs(n, H, W, seed, sigma=3.0, amp=1000.0, bg=10.0, spread=2.0, u16=False):
    """Adjoint workload: a noise-free spot reference, Poisson frames at uniform shifts."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(-spread, spread, size=(n, 2))
    ref = synth.gaussian_spot(H, W, H / 2, W / 2, sigma, amp, bg)
    frames = np.array([rng.poisson(synth.gaussian_spot(H, W, H / 2 + p[0], W / 2 + p[1], sigma, amp, bg))
                       for p in d])
    frames = frames.astype(np.uint16) if u16 else frames.astype(np.float32)
    return frames, ref.astype(np.float32), d


def to_device(torch, frames):
    if frames.dtype == np.uint16:
        return torch.from_numpy(frames.view(np.int16)).cuda().view(torch.uint16)
    return torch.from_numpy(frames).cuda()


def gpu_run(torch, frames, ref, u, method, g=None, max_batch=256):
    n, H, W = frames.shape
    t = C.Tracker(ref, upsample=u, method=method, in_dtype="u16" if frames.dtype == np.uint16 else "f32",
                  max_batch=max_batch)
    dev = to_device(torch, frames)
    rec = t.empty_results(n)
    for s in range(0, n, max_batch):
        e = min(n, s + max_batch)
        C.ccst_track(t.ctx, dev[s:e], e - s, 0, rec[s:e])
    peak = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    status = torch.empty((n,), dtype=torch.int32, device="cuda")
    C.ccst_peak_continuous(t.ctx, dev, n, 0, rec, peak, status)
    out = {"rec": None, "peak": None, "status": None, "gI": None, "gE": None}
    if g is not None:
        gd = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float32)).cuda()
        gI = torch.empty((n, H, W), dtype=torch.float32, device="cuda")
        gE = torch.empty((H, W), dtype=torch.float32, device="cuda")
        C.ccst_backward(t.ctx, dev, n, 0, rec, gd, gI, gE)
    C.ccst_sync(t.ctx)
    out["rec"] = C.decode(rec)
    out["peak"] = peak.cpu().numpy()
    out["status"] = status.cpu().numpy()
    if g is not None:
        out["gI"] = gI.cpu().numpy()
        out["gE"] = gE.cpu().numpy()
    t.close()
    return out


def oracle_seed(f, ref64, u, method, rec):
    """The oracle's own grid peak (dy, dx), from which its Newton iteration starts; the GPU
    record must match it (integer peak identical, |d| within 1e-3 px)."""
    o = oracle.track_one(f, ref64, u, method)
    assert (int(rec["ipy"]), int(rec["ipx"])) == (o["ipy"], o["ipx"]), (rec, o)
    assert abs(float(rec["dx"]) - o["dx32"]) <= 1e-3 and abs(float(rec["dy"]) - o["dy32"]) <= 1e-3, (rec, o)
    return (o["dy"], o["dx"])


def check(frames, ref, u, method, got, g=None):
    ref64 = ref.astype(np.float64)
    gE_sum = np.zeros_like(ref64)
    for i, f in enumerate(frames.astype(np.float64)):
        rec = got["rec"][i]
        pk = ad.continuous_peak(f, ref64, oracle_seed(f, ref64, u, method, rec), method)
        assert pk["ok"] and got["status"][i] == 0, (i, pk, got["status"][i])
        assert abs(got["peak"][i, 0] - pk["s"][1]) < 1e-9 and abs(got["peak"][i, 1] - pk["s"][0]) < 1e-9, \
            (i, got["peak"][i], pk["s"])
        if g is not None:
            gI, gE = ad.vjp(f, ref64, pk["s"], pk["hess"], (g[i, 1], g[i, 0]), method)
            assert np.max(np.abs(got["gI"][i] - gI)) <= 2e-6 * np.abs(gI).max(), i
            gE_sum += gE
    if g is not None:
        assert np.max(np.abs(got["gE"] - gE_sum)) <= 2e-6 * np.abs(gE_sum).max()


@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_continuous_peak_and_vjp_64x64(torch, method):
    frames, ref, _ = pairs(40, 64, 64, seed=1)
    g = np.random.default_rng(2).normal(size=(40, 2))
    got = gpu_run(torch, frames, ref, 100, method, g)
    check(frames, ref, 100, method, got, g)


@pytest.mark.parametrize("H,W,u,n,u16", [(32, 16, 37, 12, True), (16, 32, 50, 10, False), (128, 128, 100, 6, True),
                                         (8, 8, 20, 5, False)])
def test_shapes(torch, H, W, u, n, u16):
    frames, ref, _ = pairs(n, H, W, seed=H + W, sigma=min(H, W) / 10 + 0.8, spread=min(H, W) / 16, u16=u16)
    g = np.random.default_rng(3).normal(size=(n, 2))
    for method in (oracle.CC_U, oracle.CC_SN):
        got = gpu_run(torch, frames, ref, u, method, g)
        check(frames, ref, u, method, got, g)


def test_more_frames_than_ctas_sum_the_reference_gradient(torch):
    frames, ref, _ = pairs(400, 32, 32, seed=4, sigma=2.5, spread=1.5)
    g = np.random.default_rng(5).normal(size=(400, 2))
    got = gpu_run(torch, frames, ref, 50, oracle.CC_U, g, max_batch=128)
    check(frames, ref, 50, oracle.CC_U, got, g)


def test_peak_only_and_zero_frames(torch):
    frames, ref, _ = pairs(3, 32, 32, seed=6)
    t = C.Tracker(ref, upsample=50, in_dtype="f32")
    dev = to_device(torch, frames)
    rec = t.empty_results(3)
    C.ccst_track(t.ctx, dev, 3, 0, rec)
    st = torch.full((3,), -1, dtype=torch.int32, device="cuda")
    C.ccst_peak_continuous(t.ctx, dev, 3, 0, rec, None, st)        # status only
    gE = torch.full((32, 32), 7.0, dtype=torch.float32, device="cuda")
    gd = torch.zeros((0, 2), dtype=torch.float32, device="cuda")
    C.ccst_backward(t.ctx, dev, 0, 0, rec, gd, None, gE)            # no frames: dL/dE = 0
    C.ccst_sync(t.ctx)
    assert st.cpu().tolist() == [0, 0, 0] and float(gE.abs().max()) == 0.0
    with pytest.raises(C.CcstError):
        C.ccst_peak_continuous(t.ctx, dev, 3, 0, rec, None, None)  # no output
    with pytest.raises(C.CcstError):
        C.ccst_backward(t.ctx, dev, 3, 0, None, gd, None, gE)       # no records
    with pytest.raises(C.CcstError):
        C.ccst_backward(t.ctx, dev, -1, 0, rec, gd, None, gE)
    t.close()


def test_autograd_function_matches_oracle(torch):
    from paper_2310_08770_b300.autograd import continuous_peak
    frames, ref, _ = pairs(8, 64, 64, seed=7)
    t = C.Tracker(ref, upsample=100, in_dtype="f32")
    fr = torch.from_numpy(frames).cuda().requires_grad_(True)
    rf = torch.from_numpy(ref).cuda().requires_grad_(True)
    peak, status = continuous_peak(t, fr, rf)
    loss = (peak[:, 0] * 0.5 - peak[:, 1] * 1.5).sum() + (peak ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0] * 8
    p = peak.detach().cpu().numpy()
    gI = fr.grad.cpu().numpy()
    gE = rf.grad.cpu().numpy()
    t.close()
    gE_sum = np.zeros((64, 64))
    for i in range(8):
        o = oracle.track_one(frames[i].astype(np.float64), ref.astype(np.float64), 100)
        pk = ad.continuous_peak(frames[i].astype(np.float64), ref.astype(np.float64), (o["dy"], o["dx"]))
        assert abs(p[i, 0] - pk["s"][1]) < 1e-9 and abs(p[i, 1] - pk["s"][0]) < 1e-9, (p[i], pk["s"])
        gdx, gdy = 0.5 + 2 * pk["s"][1], -1.5 + 2 * pk["s"][0]
        a, b = ad.vjp(frames[i].astype(np.float64), ref.astype(np.float64), pk["s"], pk["hess"], (gdy, gdx))
        assert np.max(np.abs(gI[i] - a)) <= 2e-6 * np.abs(a).max()
        gE_sum += b
    assert np.max(np.abs(gE - gE_sum)) <= 2e-6 * np.abs(gE_sum).max()
