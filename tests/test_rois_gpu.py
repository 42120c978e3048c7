"""Uneven-ROI batches (ccst_add_reference / ccst_track_rois): ROIs of mixed sizes, each
against its own reference, in one persistent launch.

Every record must be bit-identical to ccst_track's on a context made for that ROI's
reference (the same per-frame code runs), and meet the parity bar against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
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


def uneven(n, sides, seed, u16=False):
    """ROIs with sides drawn from `sides`: per-ROI noise-free reference (random sigma, peak,
    background), Poisson frame at a uniform shift in [-3, 3] px."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        N = int(rng.choice(sides))
        sigma, amp, bg = rng.uniform(1.5, 4.0), rng.uniform(200, 5000), rng.uniform(5, 50)
        d = rng.uniform(-3, 3, size=2) * min(1.0, N / 32)
        ref = synth.gaussian_spot(N, N, N / 2, N / 2, sigma, amp, bg)
        frame = rng.poisson(synth.gaussian_spot(N, N, N / 2 + d[0], N / 2 + d[1], sigma, amp, bg))
        out.append((ref.astype(np.float32), frame.astype(np.uint16 if u16 else np.float32)))
    return out


def dev(torch, a):
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).cuda().view(torch.uint16)
    return torch.from_numpy(a).cuda()


def run_rois(torch, items, u, method=0, pad=0, u16=False):
    ref0 = items[0][0]
    t = C.Tracker(ref0, upsample=u, method=method, in_dtype="u16" if u16 else "f32")
    ids = [0] + [C.ccst_add_reference(t.ctx, r, r.shape[0], r.shape[1]) for r, _ in items[1:]]
    frames = []
    for _, f in items:
        if pad:
            buf = np.zeros((f.shape[0], f.shape[1] + pad), f.dtype)
            buf[:, :f.shape[1]] = f
            frames.append(dev(torch, buf)[:, :f.shape[1]])
        else:
            frames.append(dev(torch, f))
    rois = C.make_rois(frames, ids)
    out = t.empty_results(len(items))
    C.ccst_track_rois(t.ctx, rois, len(items), out)
    C.ccst_sync(t.ctx)
    res = C.decode(out)
    t.close()
    return res


def single(torch, ref, frame, u, method=0, u16=False):
    t = C.Tracker(ref, upsample=u, method=method, in_dtype="u16" if u16 else "f32", max_batch=1)
    out = t.empty_results(1)
    C.ccst_track(t.ctx, dev(torch, frame[None]), 1, 0, out)
    C.ccst_sync(t.ctx)
    r = C.decode(out)
    t.close()
    return r[0]


@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_rois_equal_per_reference_contexts_and_the_oracle(torch, method):
    items = uneven(40, [16, 32, 64, 128], seed=1 + method)
    res = run_rois(torch, items, 100, method)
    bad = []
    for i, ((ref, frame), g) in enumerate(zip(items, res)):
        s = single(torch, ref, frame, 100, method)
        assert g.tobytes() == s.tobytes(), (i, g, s)
        o = oracle.track_one(frame.astype(np.float64), ref.astype(np.float64), 100, method)
        int_ok = (g["ipy"], g["ipx"]) == (o["ipy"], o["ipx"]) or o["int_margin"] < TIE
        sub_ok = (abs(g["dx"] - o["dx32"]) <= TOL_PX and abs(g["dy"] - o["dy32"]) <= TOL_PX) or o["sub_margin"] < TIE
        if not (int_ok and sub_ok):
            bad.append(i)
    assert not bad, bad


@pytest.mark.parametrize("u", [7, 120, 200])
def test_rois_upsampling_factors(torch, u):
    # the 128 px class across its plans: tcgen05 at u = 7 (one chunk), the warp-MMA stages
    # in chunks at u = 120, the stage tables read from global memory at u = 200 (the
    # 128 x 128 ROI kernel with both contraction forms); every record equals its own
    # context's
    items = uneven(12, [16, 64, 128], seed=20 + u)
    res = run_rois(torch, items, u)
    for i, ((ref, frame), g) in enumerate(zip(items, res)):
        assert g.tobytes() == single(torch, ref, frame, u).tobytes(), (u, i)


def test_rois_u16_padded_rows_and_many_items(torch):
    items = uneven(300, [32, 64], seed=5, u16=True)
    res = run_rois(torch, items, 50, pad=8, u16=True)
    for i in (0, 1, 2, 150, 298, 299):
        ref, frame = items[i]
        assert res[i].tobytes() == single(torch, ref, frame, 50, u16=True).tobytes(), i


def test_rois_errors(torch):
    ref = synth.gaussian_spot(32, 32, 16, 16, 2.0, 800.0, 10.0).astype(np.float32)
    t = C.Tracker(ref, upsample=20, in_dtype="f32")
    with pytest.raises(C.CcstError) as e:
        C.ccst_add_reference(t.ctx, np.zeros((300, 300), np.float32), 300, 300)   # above 256
    assert e.value.code == C.E_SHAPE
    with pytest.raises(C.CcstError):
        C.ccst_add_reference(t.ctx, np.zeros((32, 64), np.float32), 32, 64)   # not square
    r1 = C.ccst_add_reference(t.ctx, np.zeros((64, 64), np.float32) + 5, 64, 64)
    f32 = torch.zeros((32, 32), dtype=torch.float32, device="cuda")
    f64 = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    out = t.empty_results(2)
    C.ccst_track_rois(t.ctx, C.make_rois([f32], [0]), 0, out)                 # n = 0
    with pytest.raises(C.CcstError) as e:
        C.ccst_track_rois(t.ctx, C.make_rois([f32], [r1]), 1, out)           # size differs
    assert e.value.code == C.E_SHAPE
    with pytest.raises(C.CcstError):
        C.ccst_track_rois(t.ctx, C.make_rois([f32], [7]), 1, out)            # unknown id
    C.ccst_track_rois(t.ctx, C.make_rois([f32, f64], [0, r1]), 2, out)
    C.ccst_sync(t.ctx)
    t.close()
