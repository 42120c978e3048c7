"""Real-time reference (Sec. III B, Eq. (9)) and drift removal (Eqs. (10)-(12)) through the
C ABI, against the FP64 oracle (``oracle.rt_oracle``).

Bar, as for the fixed reference: integer peaks identical and |dx|, |dy| within 1e-3 px of
the oracle, a frame whose oracle top-2 margin is below 1e-12 (a genuine tie) excepted. The
GPU's filtered reference differs from the oracle's by FP64 rounding only, so every frame
is held to that bar against the oracle's own reference at that frame.
"""
import numpy as np
import pytest

import oracle
from oracle import rt_oracle as rt
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


def spot_stream(n, H, W, step, seed, sigma=2.0, amp=800.0, bg=10.0, u16=True):
    """A spot on a random walk (start at the centre), Poisson frames."""
    rng = np.random.default_rng(seed)
    pos = np.cumsum(rng.normal(0, step, size=(n, 2)), axis=0)
    pos -= pos[0]
    frames = np.array([rng.poisson(synth.gaussian_spot(H, W, H / 2 + p[0], W / 2 + p[1], sigma, amp, bg))
                       for p in pos])
    return (frames.astype(np.uint16) if u16 else frames.astype(np.float32)), pos


def to_device(torch, frames):
    if frames.dtype == np.uint16:
        return torch.from_numpy(frames.view(np.int16)).cuda().view(torch.uint16)
    return torch.from_numpy(frames).cuda()


def rt_gpu(torch, frames, u, a0, b1=None, method=0, eps=200.0, splits=()):
    """ccst_rt_begin on frames[0], then ccst_rt_track over frames[1:] (in pieces at `splits`)."""
    n, H, W = frames.shape
    t = C.Tracker(np.zeros((H, W), np.float32), upsample=u, method=method, eps=eps,
                  in_dtype="u16" if frames.dtype == np.uint16 else "f32")
    dev = to_device(torch, frames)
    torch.cuda.synchronize()
    b1 = 1.0 - a0 if b1 is None else b1
    C.ccst_rt_begin(t.ctx, dev[0], 0, a0, b1)
    out = t.empty_results(n - 1)
    cuts = [1, *splits, n]
    for s, e in zip(cuts[:-1], cuts[1:]):
        C.ccst_rt_track(t.ctx, dev[s:e], e - s, 0, out[s - 1:e - 1])
    C.ccst_sync(t.ctx)
    res = C.decode(out)
    t.close()
    return res


def compare(res, orc):
    bad = []
    for i, (g, o) in enumerate(zip(res, orc)):
        int_ok = (g["ipy"], g["ipx"]) == (o["ipy"], o["ipx"]) or o["int_margin"] < TIE
        sub_ok = (abs(g["dx"] - o["dx32"]) <= TOL_PX and abs(g["dy"] - o["dy32"]) <= TOL_PX) or \
            o["sub_margin"] < TIE
        if not (int_ok and sub_ok):
            bad.append((i, (g["ipy"], g["ipx"], g["dx"], g["dy"]), (o["ipy"], o["ipx"], o["dx32"], o["dy32"])))
    assert not bad, f"{len(bad)} of {len(res)} frames differ, first: {bad[:3]}"


@pytest.mark.parametrize("H,W,u,a0,n,step,u16", [
    (64, 64, 100, 0.2, 24, 0.4, True),
    (128, 128, 100, 0.05, 16, 0.3, True),
    (32, 16, 37, 1.0, 12, 0.5, False),     # memoryless filter: E_i is the aligned frame i
    (16, 32, 1, 0.5, 10, 0.8, False),      # u = 1: whole-pixel displacements only
])
def test_rt_track_matches_oracle_ccu(torch, H, W, u, a0, n, step, u16):
    frames, _ = spot_stream(n, H, W, step, seed=H + W + u, u16=u16)
    orc = rt.rt_track(frames.astype(np.float64), u=u, a0=a0, method=oracle.CC_U)
    compare(rt_gpu(torch, frames, u, a0), orc)


# extreme aspect ratios: the update's cooperative grid is max(H/2, W/2 + 1) CTAs, and the
# narrow shapes take the plain-FP32 contraction stages
@pytest.mark.parametrize("H,W", [(8, 8), (128, 8), (8, 128), (128, 32), (16, 64)])
def test_rt_track_shapes(torch, H, W):
    frames, _ = spot_stream(10, H, W, 0.3, seed=3 * H + W, sigma=1.5)
    orc = rt.rt_track(frames.astype(np.float64), u=50, a0=0.3, method=oracle.CC_U)
    compare(rt_gpu(torch, frames, 50, 0.3), orc)


@pytest.mark.parametrize("H,W,u,a0,n", [(64, 64, 100, 0.2, 16), (32, 32, 50, 0.5, 12)])
def test_rt_track_matches_oracle_ccsn(torch, H, W, u, a0, n):
    frames, _ = spot_stream(n, H, W, 0.4, seed=7 * H + u)
    orc = rt.rt_track(frames.astype(np.float64), u=u, a0=a0, method=oracle.CC_SN, eps=200.0)
    compare(rt_gpu(torch, frames, u, a0, method=oracle.CC_SN), orc)


def test_rt_frozen_filter_tracks_against_frame_zero(torch):
    # a0 = 0, b1 = 1: the reference stays E_0 = I_0, the fixed-reference path with ref = frame 0
    frames, _ = spot_stream(20, 64, 64, 0.5, seed=11)
    orc = oracle.track_batch(frames[1:].astype(np.float64), frames[0].astype(np.float64), u=100,
                             method=oracle.CC_U)
    compare(rt_gpu(torch, frames, 100, 0.0, b1=1.0), orc)


def test_rt_calls_continue_the_filter(torch):
    # the filter state lives in the context: split calls give the records of one call, bit for bit
    frames, _ = spot_stream(14, 32, 32, 0.4, seed=12)
    one = rt_gpu(torch, frames, 50, 0.3)
    split = rt_gpu(torch, frames, 50, 0.3, splits=(2, 3, 9))
    assert one.tobytes() == split.tobytes()


def test_rt_low_pass_reference_follows_the_spot(torch):
    frames, pos = spot_stream(40, 64, 64, 0.3, seed=13, sigma=2.5, amp=2000.0, bg=20.0)
    res = rt_gpu(torch, frames, 100, 0.1)
    err = np.hypot(res["dx"] - pos[1:, 1], res["dy"] - pos[1:, 0])
    assert err.max() < 0.15


def test_rt_errors(torch):
    t = C.Tracker(np.zeros((16, 16), np.float32), upsample=10, in_dtype="f32")
    dev = torch.zeros((3, 16, 16), dtype=torch.float32, device="cuda")
    out = t.empty_results(3)
    with pytest.raises(C.CcstError) as e:
        C.ccst_rt_track(t.ctx, dev, 3, 0, out)         # no ccst_rt_begin yet
    assert e.value.code == C.E_INVALID
    with pytest.raises(C.CcstError):
        C.ccst_rt_begin(t.ctx, dev[0], 0, float("nan"), 0.5)
    with pytest.raises(C.CcstError):
        C.ccst_rt_begin(t.ctx, dev[0], 8, 0.1, 0.9)    # pitch < W
    C.ccst_rt_begin(t.ctx, dev[0], 0, 0.1, 0.9)
    C.ccst_rt_track(t.ctx, dev, 0, 0, out)               # n = 0: nothing to do
    with pytest.raises(C.CcstError):
        C.ccst_rt_track(t.ctx, dev, -1, 0, out)
    C.ccst_rt_track(t.ctx, dev, 3, 0, out)
    C.ccst_sync(t.ctx)
    t.close()


def _records(torch, r):
    rec = np.zeros(len(r), dtype=C.RESULT_DTYPE)
    rec["dx"], rec["dy"] = r[:, 0], r[:, 1]
    return torch.from_numpy(rec.view(np.uint8).reshape(len(r), 24).copy()).cuda()


@pytest.mark.parametrize("alpha", [0.0, 0.5, 5.0])
def test_drift_correct_matches_oracle(torch, alpha):
    rng = np.random.default_rng(21)
    n, a0, u = 3000, 0.02, 100
    # a slow ramp plus jitter, and a jump that the rate limit holds back
    r = np.linspace(0, 3, n)[:, None] * np.array([1.0, -0.5]) + rng.normal(0, 0.05, (n, 2))
    r[n // 2:] += np.array([4.0, 3.0])
    r = r.astype(np.float32).astype(np.float64)          # the records carry float32
    dev = _records(torch, r)
    out = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    C.ccst_drift_correct(dev, n, a0, 1 - a0, alpha, u, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = rt.drift_filter(r, a0, 1 - a0) if alpha <= 0 else rt.drift_filter_limited(r, a0, 1 - a0, alpha, u)
    assert np.allclose(got, want, rtol=0, atol=1e-12)


def test_drift_correct_errors(torch):
    dev = _records(torch, np.zeros((4, 2)))
    out = torch.empty((4, 2), dtype=torch.float64, device="cuda")
    C.ccst_drift_correct(dev, 0, 0.1, 0.9, 0.0, 100, out)
    for args in [(-1, 0.1, 0.9, 0.0, 100), (4, float("inf"), 0.9, 0.0, 100), (4, 0.1, 0.9, 0.5, 0)]:
        with pytest.raises(C.CcstError):
            C.ccst_drift_correct(dev, *args, out)


def test_rt_bounded_barrier_marks_records_stale_and_begin_recovers(torch):
    # the update's grid barriers wait for one CTA too many: every wait runs out, the record
    # and all later ones carry CCST_R_RT_STALE, and ccst_rt_begin starts afresh
    frames, _ = spot_stream(6, 32, 32, 0.4, seed=14)
    fresh = rt_gpu(torch, frames, 20, 0.3)
    t = C.Tracker(np.zeros((32, 32), np.float32), upsample=20, in_dtype="u16")
    dev = to_device(torch, frames)
    out = t.empty_results(5)
    with pytest.raises(C.CcstError):
        C.ccst_debug_rt_timeout(t.ctx, dev[1], 0, out[0:1])      # no ccst_rt_begin yet
    C.ccst_rt_begin(t.ctx, dev[0], 0, 0.3, 0.7)
    C.ccst_rt_track(t.ctx, dev[1:3], 2, 0, out[0:2])
    C.ccst_debug_rt_timeout(t.ctx, dev[2], 0, out[1:2])
    C.ccst_rt_track(t.ctx, dev[3:6], 3, 0, out[2:5])
    C.ccst_sync(t.ctx)
    r = C.decode(out)
    stale = (r["flags"] & C.R_RT_STALE) != 0
    assert stale.tolist() == [False, True, True, True, True]
    # frame 2 was tracked before its update failed: its record matches the undisturbed run
    assert r[1]["ipy"] == fresh[1]["ipy"] and r[1]["dx"] == fresh[1]["dx"]
    C.ccst_rt_begin(t.ctx, dev[0], 0, 0.3, 0.7)
    C.ccst_rt_track(t.ctx, dev[1:6], 5, 0, out)
    C.ccst_sync(t.ctx)
    assert C.decode(out).tobytes() == fresh.tobytes()
    t.close()
