"""Offline iterative reference (Sec. III A, Eq. (8)) through the C ABI, against the FP64
oracle (``oracle.offline_oracle``).

Per pass: the records of every frame meet the fixed-reference bar (integer peaks identical,
|dx|, |dy| within 1e-3 px, genuine ties excepted) against the oracle's own E_n, and the
context's FP64 reference operand matches the oracle's E_n (CC-SN: 1/(E_n + eps)) to
1e-12 of its largest value: the sums differ from the oracle's only in rounding order.
"""
import numpy as np
import pytest

import oracle
from oracle import offline_oracle as off
from paper_2310_08770_b300 import ccst as C
from paper_2310_08770_b300 import synth

pytestmark = pytest.mark.gpu

TOL_PX = 1e-3
TIE = 1e-12


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08770_b300 import build
    build.build()
    return _t


def spot_frames(n, H, W, seed, spread=2.0, sigma=2.0, amp=600.0, bg=15.0, u16=True):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-spread, spread, size=(n, 2))
    pos[0] = 0
    frames = np.array([rng.poisson(synth.gaussian_spot(H, W, H / 2 + p[0], W / 2 + p[1], sigma, amp, bg))
                       for p in pos])
    return frames.astype(np.uint16) if u16 else frames.astype(np.float32)


def to_device(torch, frames):
    if frames.dtype == np.uint16:
        return torch.from_numpy(frames.view(np.int16)).cuda().view(torch.uint16)
    return torch.from_numpy(frames).cuda()


def compare(res, orc):
    bad = []
    for i, (g, o) in enumerate(zip(res, orc)):
        int_ok = (g["ipy"], g["ipx"]) == (o["ipy"], o["ipx"]) or o["int_margin"] < TIE
        sub_ok = (abs(g["dx"] - o["dx32"]) <= TOL_PX and abs(g["dy"] - o["dy32"]) <= TOL_PX) or \
            o["sub_margin"] < TIE
        if not (int_ok and sub_ok):
            bad.append((i, (g["ipy"], g["ipx"], g["dx"], g["dy"]), (o["ipy"], o["ipx"], o["dx32"], o["dy32"])))
    assert not bad, f"{len(bad)} of {len(res)} frames differ, first: {bad[:3]}"


def stepwise(torch, frames, u, passes, method=0, eps=200.0, max_batch=64):
    """set_reference_frame, then per pass: track all frames in batches, Eq. (8) update. Returns
    the records and the reference operands of every pass."""
    n, H, W = frames.shape
    t = C.Tracker(np.zeros((H, W), np.float32), upsample=u, method=method, eps=eps, max_batch=max_batch,
                  in_dtype="u16" if frames.dtype == np.uint16 else "f32")
    dev = to_device(torch, frames)
    out = t.empty_results(n)
    refbuf = torch.empty((H, W), dtype=torch.float64, device="cuda")
    recs, refs = [], []
    C.ccst_set_reference_frame(t.ctx, dev[0])
    for p in range(passes + 1):
        for s in range(0, n, max_batch):
            e = min(n, s + max_batch)
            C.ccst_track(t.ctx, dev[s:e], e - s, 0, out[s:e])
        C.ccst_debug_reference(t.ctx, refbuf)
        C.ccst_sync(t.ctx)
        recs.append(C.decode(out).copy())
        refs.append(refbuf.cpu().numpy())
        if p < passes:
            C.ccst_offline_update(t.ctx, dev, n, 0, out)
    assert not C.ccst_reference_status(t.ctx)
    t.close()
    return recs, refs


def check_refs(refs, orefs, method, eps=200.0):
    for n, (g, E) in enumerate(zip(refs, orefs)):
        want = E if method == oracle.CC_U else 1.0 / (E + eps)
        assert np.max(np.abs(g - want)) <= 1e-12 * np.max(np.abs(want)), f"reference of pass {n}"


@pytest.mark.parametrize("H,W,u,n,passes,u16", [
    (64, 64, 100, 40, 3, True),
    (32, 16, 37, 300, 2, False),       # more frames than SMs: several frames per CTA
    (128, 128, 100, 24, 2, True),
    (16, 32, 1, 20, 2, True),          # u = 1: whole pixels
])
def test_offline_passes_match_oracle_ccu(torch, H, W, u, n, passes, u16):
    frames = spot_frames(n, H, W, seed=H * W + n, u16=u16)
    res, refs = stepwise(torch, frames, u, passes)
    ores, orefs = off.offline_track(frames.astype(np.float64), u=u, passes=passes)
    check_refs(refs, orefs, oracle.CC_U)
    for p in range(passes + 1):
        compare(res[p], ores[p])


# extreme aspect ratios (the accumulation's grid follows the frame shape; the narrow shapes
# take the plain-FP32 contraction stages)
@pytest.mark.parametrize("H,W", [(8, 8), (128, 8), (8, 128), (128, 32)])
def test_offline_shapes(torch, H, W):
    frames = spot_frames(24, H, W, seed=5 * H + W, u16=True)
    res, refs = stepwise(torch, frames, 50, 2)
    ores, orefs = off.offline_track(frames.astype(np.float64), u=50, passes=2)
    check_refs(refs, orefs, oracle.CC_U)
    for p in range(3):
        compare(res[p], ores[p])


@pytest.mark.parametrize("H,W,u,n,passes", [(64, 64, 100, 32, 2), (32, 32, 50, 200, 3)])
def test_offline_passes_match_oracle_ccsn(torch, H, W, u, n, passes):
    frames = spot_frames(n, H, W, seed=3 * n + u)
    res, refs = stepwise(torch, frames, u, passes, method=oracle.CC_SN)
    ores, orefs = off.offline_track(frames.astype(np.float64), u=u, passes=passes, method=oracle.CC_SN)
    check_refs(refs, orefs, oracle.CC_SN)
    for p in range(passes + 1):
        compare(res[p], ores[p])


def test_offline_track_is_the_stepwise_last_pass(torch):
    frames = spot_frames(150, 32, 32, seed=31)
    res, _ = stepwise(torch, frames, 50, 3, max_batch=64)
    t = C.Tracker(np.zeros((32, 32), np.float32), upsample=50, in_dtype="u16", max_batch=64)
    got = t.offline_track(to_device(torch, frames), passes=3)
    t.close()
    assert got.tobytes() == res[3].tobytes()


def test_single_frame_dataset_is_a_fixed_point(torch):
    frames = spot_frames(1, 32, 32, seed=32)
    res, refs = stepwise(torch, frames, 50, 2)
    assert all((r[0]["dx"], r[0]["dy"]) == (0.0, 0.0) for r in res)
    assert np.allclose(refs[2], refs[0], rtol=0, atol=1e-12 * np.abs(refs[0]).max())


def test_offline_errors(torch):
    t = C.Tracker(np.zeros((16, 16), np.float32), upsample=10, in_dtype="f32")
    dev = torch.zeros((3, 16, 16), dtype=torch.float32, device="cuda")
    out = t.empty_results(3)
    C.ccst_offline_update(t.ctx, dev, 0, 0, out)                  # n = 0: nothing to do
    for args in [(-1, 0, out), (3, 8, out), (3, 0, None)]:
        with pytest.raises(C.CcstError):
            C.ccst_offline_update(t.ctx, dev, *args)
    for n, passes in [(0, 1), (3, -1)]:
        with pytest.raises(C.CcstError):
            C.ccst_offline_track(t.ctx, dev, n, 0, passes, out)
    with pytest.raises(C.CcstError):
        C.ccst_set_reference_frame(t.ctx, None)
    t.close()
