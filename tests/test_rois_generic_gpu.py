"""The general-size path of uneven-ROI batches (sides other than 16, 32, 64, 128): the FP32
general-size kernel for 48, 96, 192 and 256 with the double-float kernel behind it, and the
double-float kernel alone for every other side, launched beside the power-of-two kernel by
the same ccst_track_rois call. Records must meet the FP64 oracle's parity bar (integer peaks
equal, |dx|, |dy| within 1e-3 px, genuine ties excepted) and carry CCST_R_FP32_GENERAL or
CCST_R_GENERIC; a ROI gives the same record alone and in a mixed batch."""
import numpy as np
import pytest

import oracle
from paper_2310_08770_b300 import ccst as C
from paper_2310_08770_b300 import synth

pytestmark = pytest.mark.gpu

TOL_PX = 1e-3
TIE = 1e-12
POW2 = (16, 32, 64, 128)


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08770_b300 import build
    build.build()
    return _t


def uneven(sides, seed, u16=False):
    rng = np.random.default_rng(seed)
    out = []
    for N in sides:
        sigma, amp, bg = rng.uniform(1.5, 3.5), rng.uniform(300, 4000), rng.uniform(5, 40)
        d = rng.uniform(-2, 2, size=2) * min(1.0, N / 24)
        ref = synth.gaussian_spot(N, N, N / 2, N / 2, sigma, amp, bg)
        frame = rng.poisson(synth.gaussian_spot(N, N, N / 2 + d[0], N / 2 + d[1], sigma, amp, bg))
        out.append((ref.astype(np.float32), frame.astype(np.uint16 if u16 else np.float32)))
    return out


def dev(torch, a):
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).cuda().view(torch.uint16)
    return torch.from_numpy(a).cuda()


def run(torch, items, u, method=0, u16=False):
    t = C.Tracker(synth.gaussian_spot(32, 32, 16, 16, 2.0, 500.0, 10.0).astype(np.float32), upsample=u,
                  method=method, in_dtype="u16" if u16 else "f32")
    ids = [C.ccst_add_reference(t.ctx, r, *r.shape) for r, _ in items]
    frames = [dev(torch, f) for _, f in items]
    out = t.empty_results(len(items))
    C.ccst_track_rois(t.ctx, C.make_rois(frames, ids), len(items), out)
    C.ccst_sync(t.ctx)
    res = C.decode(out)
    t.close()
    return res


def check(items, res, u, method):
    bad = []
    for i, ((ref, frame), g) in enumerate(zip(items, res)):
        N = ref.shape[0]
        assert bool(g["flags"] & (C.R_GENERIC | C.R_FP32_GENERAL)) == (N not in POW2), (i, N, g["flags"])
        o = oracle.track_one(frame.astype(np.float64), ref.astype(np.float64), u, method)
        int_ok = (g["ipy"], g["ipx"]) == (o["ipy"], o["ipx"]) or o["int_margin"] < TIE
        sub_ok = (abs(g["dx"] - o["dx32"]) <= TOL_PX and abs(g["dy"] - o["dy32"]) <= TOL_PX) or o["sub_margin"] < TIE
        if not (int_ok and sub_ok):
            bad.append((i, N, (g["ipy"], g["ipx"], g["dx"], g["dy"]), (o["ipy"], o["ipx"], o["dx32"], o["dy32"])))
        if N not in POW2:
            assert abs(g["peak"] - o["peak"]) <= 1e-5 * abs(o["peak"]) + 1e-30, (i, g["peak"], o["peak"])
    assert not bad, bad


@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_general_sides_mixed_with_power_of_two_match_the_oracle(torch, method):
    items = uneven([48, 96, 32, 8, 24, 64, 48, 30, 96, 16, 12, 40], seed=10 + method)
    res = run(torch, items, 100, method)
    check(items, res, 100, method)


def test_large_general_sides(torch):
    items = uneven([192, 256, 144], seed=20, u16=True)
    res = run(torch, items, 50, u16=True)
    check(items, res, 50, oracle.CC_U)


def test_general_roi_alone_and_in_a_batch(torch):
    items = uneven([96, 48, 64, 96, 24], seed=30)
    mixed = run(torch, items, 100)
    for k in (0, 1, 4):
        alone = run(torch, [items[k]], 100)
        assert alone[0].tobytes() == mixed[k].tobytes(), k


def test_general_size_errors(torch):
    t = C.Tracker(np.ones((32, 32), np.float32), upsample=20, in_dtype="f32")
    for N in (4, 300):
        with pytest.raises(C.CcstError) as e:
            C.ccst_add_reference(t.ctx, np.ones((N, N), np.float32), N, N)
        assert e.value.code == C.E_SHAPE
    r48 = C.ccst_add_reference(t.ctx, np.ones((48, 48), np.float32) * 3, 48, 48)
    f96 = dev(torch, np.ones((96, 96), np.float32))
    out = t.empty_results(1)
    with pytest.raises(C.CcstError) as e:
        C.ccst_track_rois(t.ctx, C.make_rois([f96], [r48]), 1, out)          # size differs
    assert e.value.code == C.E_SHAPE
    t.close()


def test_graph_captured_batches_replay_the_direct_records(torch):
    # with CCST_FLAG_GRAPHS a work list is captured once per stream (all its kernels in one
    # graph) and replayed; records are byte-identical to the direct path's, every record is
    # written on every replay, and a new reference drops the captured graphs
    items = uneven([48, 32, 96, 64, 24, 128, 48, 16, 96, 32], seed=21, u16=True)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ref0 = synth.gaussian_spot(32, 32, 16, 16, 2.0, 500.0, 10.0).astype(np.float32)
    direct = C.Tracker(ref0, upsample=60, in_dtype="u16")
    ids = [C.ccst_add_reference(direct.ctx, r, *r.shape) for r, _ in items]
    frames = [dev(torch, f) for _, f in items]
    want = direct.empty_results(len(items))
    C.ccst_track_rois(direct.ctx, C.make_rois(frames, ids), len(items), want)
    C.ccst_sync(direct.ctx)
    want = C.decode(want).tobytes()
    direct.close()
    t = C.Tracker(ref0, upsample=60, in_dtype="u16", graphs=True, stream=streams[0])
    gids = [C.ccst_add_reference(t.ctx, r, *r.shape) for r, _ in items]
    rois = C.make_rois(frames, gids)
    for rep in range(3):
        for st in streams:
            C.ccst_set_stream(t.ctx, st.cuda_stream)
            out = torch.full((len(items), 24), 0xFF, dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
            C.ccst_track_rois(t.ctx, rois, len(items), out)
            torch.cuda.synchronize()
            assert C.decode(out).tobytes() == want, (rep, st)
            if rep == 0:
                keep = out          # the graph captured for this out buffer
            del out
    # the same list on the same stream and output buffer replays its graph
    out = torch.empty((len(items), 24), dtype=torch.uint8, device="cuda")
    C.ccst_set_stream(t.ctx, streams[1].cuda_stream)
    C.ccst_track_rois(t.ctx, rois, len(items), out)
    g = C.ccst_graph_stats(t.ctx)
    for _ in range(3):
        C.ccst_track_rois(t.ctx, rois, len(items), out)
    torch.cuda.synchronize()
    g2 = C.ccst_graph_stats(t.ctx)
    assert g2["instantiations"] == g["instantiations"] and g2["replays"] == g["replays"] + 3
    assert 1 <= g["cached"] <= 7
    assert C.decode(out).tobytes() == want
    C.ccst_add_reference(t.ctx, items[0][0], 48, 48)          # drops the captured graphs
    C.ccst_track_rois(t.ctx, rois, len(items), out)
    torch.cuda.synchronize()
    g3 = C.ccst_graph_stats(t.ctx)
    assert g3["cached"] == 1 and g3["instantiations"] == g2["instantiations"] + 1
    assert C.decode(out).tobytes() == want
    del keep
    t.close()


def test_power_of_two_work_list_is_captured_once(torch):
    # a list with no general-size ROI on a context without general plans: one capture, then
    # replays only
    items = uneven([32, 64, 16, 128, 32, 64], seed=23)
    t = C.Tracker(synth.gaussian_spot(32, 32, 16, 16, 2.0, 500.0, 10.0).astype(np.float32), upsample=50,
                  in_dtype="f32", graphs=True, stream=torch.cuda.Stream())
    ids = [C.ccst_add_reference(t.ctx, r, *r.shape) for r, _ in items]
    rois = C.make_rois([dev(torch, f) for _, f in items], ids)
    out = t.empty_results(len(items))
    for _ in range(5):
        C.ccst_track_rois(t.ctx, rois, len(items), out)
    C.ccst_sync(t.ctx)
    assert C.ccst_graph_stats(t.ctx) == {"instantiations": 1, "replays": 5, "cached": 1}
    t.close()
