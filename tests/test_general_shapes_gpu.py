"""General-shape contexts: ccst_create with any H, W from 8 to 256 that the power-of-two
kernel does not take (48 x 48, 96 x 96, 256 x 128, 192 x 64, 24 x 40, 100 x 60, 256 x 256).
Square sides 48, 96, 192 and 256 run on the FP32 general-size kernel (CCST_R_FP32_GENERAL),
with the double-float kernel taking the frames its guards cannot certify; every other shape
runs on the double-float kernel (CCST_R_GENERIC). Records meet the FP64 oracle's parity bar
(integer peaks equal, |dx|, |dy| within 1e-3 px, genuine ties excepted); the device, host and
ticket paths give the same records; the entry points that need the power-of-two path's
spectra refuse with CCST_E_UNSUPPORTED."""
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


def pairs(H, W, n, seed, u16):
    """Noise-free spot reference at the centre; Poisson frames shifted by U(-2, 2) px per
    axis (scaled down for frames under 24 px)."""
    rng = np.random.default_rng(seed)
    sigma, amp, bg = rng.uniform(1.8, 3.5), rng.uniform(400, 4000), rng.uniform(5, 40)
    ref = synth.gaussian_spot(H, W, H / 2, W / 2, sigma, amp, bg)
    s = min(1.0, min(H, W) / 24)
    d = rng.uniform(-2, 2, size=(n, 2)) * s
    fr = np.array([rng.poisson(synth.gaussian_spot(H, W, H / 2 + p[0], W / 2 + p[1], sigma, amp, bg)) for p in d])
    return ref.astype(np.float32), fr.astype(np.uint16 if u16 else np.float32)


def dev(torch, a, pad=0):
    if pad:
        buf = np.zeros(a.shape[:-1] + (a.shape[-1] + pad,), a.dtype)
        buf[..., :a.shape[-1]] = a
        a = buf
    t = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda()
    return t.view(torch.uint16) if a.dtype == np.uint16 else t


def wait(ctx, ticket):
    while not C.ccst_poll(ctx, ticket, 100000):
        pass


def tracker(ref, u, method, u16, max_batch=64):
    return C.Tracker(ref, upsample=u, method=method, in_dtype="u16" if u16 else "f32", max_batch=max_batch)


def track(torch, t, frames, pad=0):
    d = dev(torch, frames, pad)
    out = t.empty_results(len(frames))
    C.ccst_track(t.ctx, d, len(frames), frames.shape[-1] + pad if pad else 0, out)
    C.ccst_sync(t.ctx)
    return C.decode(out)


def check(ref, frames, res, u, method):
    bad = []
    for i, (f, g) in enumerate(zip(frames, res)):
        assert g["flags"] & (C.R_GENERIC | C.R_FP32_GENERAL), (i, g["flags"])
        o = oracle.track_one(f.astype(np.float64), ref.astype(np.float64), u, method)
        int_ok = (g["ipy"], g["ipx"]) == (o["ipy"], o["ipx"]) or o["int_margin"] < TIE
        sub_ok = (abs(g["dx"] - o["dx32"]) <= TOL_PX and abs(g["dy"] - o["dy32"]) <= TOL_PX) or o["sub_margin"] < TIE
        if not (int_ok and sub_ok):
            bad.append((i, (g["ipy"], g["ipx"], g["dx"], g["dy"]), (o["ipy"], o["ipx"], o["dx32"], o["dy32"])))
        assert abs(g["peak"] - o["peak"]) <= 1e-5 * abs(o["peak"]), (i, g["peak"], o["peak"])
    assert not bad, bad


@pytest.mark.parametrize("H,W,u,u16", [(48, 48, 100, True), (96, 96, 100, False), (256, 128, 100, True),
                                       (192, 64, 37, False), (24, 40, 100, True), (100, 60, 64, False),
                                       (9, 27, 20, True), (256, 256, 25, True)])
@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_general_shapes_match_the_oracle(torch, H, W, u, u16, method):
    ref, frames = pairs(H, W, 6 if H * W > 20000 else 12, seed=H * 1000 + W + method, u16=u16)
    t = tracker(ref, u, method, u16)
    assert C.ccst_grid_size(t.ctx) == oracle.grid_size(u)
    res = track(torch, t, frames)
    t.close()
    check(ref, frames, res, u, method)


def test_more_frames_than_ctas_and_padded_rows(torch):
    ref, frames = pairs(48, 72, 700, seed=5, u16=True)
    t = tracker(ref, 50, oracle.CC_U, True, max_batch=700)
    plain = track(torch, t, frames)
    padded = track(torch, t, frames, pad=8)
    t.close()
    assert plain.tobytes() == padded.tobytes()
    idx = [0, 1, 295, 296, 297, 591, 592, 699]
    check(ref, frames[idx], plain[idx], 50, oracle.CC_U)


def test_host_ticket_and_roi_paths_give_the_same_records(torch):
    ref, frames = pairs(96, 96, 40, seed=6, u16=True)
    t = tracker(ref, 100, oracle.CC_U, True)
    want = track(torch, t, frames)
    # blocking host path
    host = np.zeros(40, C.RESULT_DTYPE)
    C.ccst_track_host(t.ctx, frames, 40, 0, host)
    assert host.tobytes() == want.tobytes()
    # pipelined host path: four submissions in flight over the two internal streams
    outs = [np.zeros(10, C.RESULT_DTYPE) for _ in range(4)]
    tickets = [C.ccst_submit_host(t.ctx, frames[10 * k:10 * (k + 1)], 10, 0, outs[k]) for k in range(4)]
    for tk in tickets:
        wait(t.ctx, tk)
    assert np.concatenate(outs).tobytes() == want.tobytes()
    # device tickets
    d = dev(torch, frames)
    out = t.empty_results(40)
    tk = C.ccst_submit(t.ctx, d, 40, out)
    wait(t.ctx, tk)
    assert C.decode(out).tobytes() == want.tobytes()
    # the context's reference (id 0) in an ROI batch, beside another general size
    r2 = C.ccst_add_reference(t.ctx, ref[:48, :48].copy(), 48, 48)
    f2 = dev(torch, frames[:, :48, :48].copy())
    out2 = t.empty_results(8)
    C.ccst_track_rois(t.ctx, C.make_rois([d[i] for i in range(4)] + [f2[i] for i in range(4)], [0] * 4 + [r2] * 4),
                      8, out2)
    C.ccst_sync(t.ctx)
    got = C.decode(out2)
    t.close()
    assert got[:4].tobytes() == want[:4].tobytes()


def test_frame_set_as_reference(torch):
    ref, frames = pairs(60, 60, 9, seed=7, u16=True)
    t = tracker(np.ones((60, 60), np.float32), 100, oracle.CC_SN, True)
    d = dev(torch, frames)
    C.ccst_set_reference_frame(t.ctx, d[0])
    out = t.empty_results(8)
    C.ccst_track(t.ctx, d[1:], 8, 0, out)
    C.ccst_sync(t.ctx)
    res = C.decode(out)
    t.close()
    check(frames[0].astype(np.float32), frames[1:], res, 100, oracle.CC_SN)


def test_power_of_two_only_entry_points_refuse(torch):
    ref, frames = pairs(48, 48, 2, seed=8, u16=False)
    t = tracker(ref, 100, oracle.CC_U, False)
    d = dev(torch, frames)
    rec = t.empty_results(2)
    C.ccst_track(t.ctx, d, 2, 0, rec)
    peak = torch.empty((2, 2), dtype=torch.float64, device="cuda")
    for call in (lambda: C.ccst_rt_begin(t.ctx, d[0], 0, 0.2, 0.8),
                 lambda: C.ccst_offline_track(t.ctx, d, 2, 0, 1, rec),
                 lambda: C.ccst_peak_continuous(t.ctx, d, 2, 0, rec, peak, None)):
        with pytest.raises(C.CcstError) as e:
            call()
        assert e.value.code == C.E_UNSUPPORTED
    C.ccst_track(t.ctx, d, 2, 0, rec)                 # the context stays usable
    C.ccst_sync(t.ctx)
    t.close()


def test_shapes_outside_the_range_are_refused(torch):
    for H, W in [(4, 64), (64, 300), (257, 8)]:
        with pytest.raises(C.CcstError) as e:
            C.Tracker(np.ones((H, W), np.float32), upsample=10, in_dtype="f32")
        assert e.value.code == C.E_SHAPE


@pytest.mark.parametrize("H,W,u,method", [(72, 72, 100, oracle.CC_U), (48, 80, 64, oracle.CC_SN),
                                          (30, 30, 100, oracle.CC_U), (192, 128, 50, oracle.CC_U),
                                          (12, 8, 3, oracle.CC_SN),
                                          # grids above 256 points a side: pass 2 recomputes the
                                          # FP32 values, and the row bitmap spans many words
                                          (40, 24, 200, oracle.CC_U), (20, 20, 1000, oracle.CC_SN)])
def test_fp32_grid_with_candidates_equals_the_exhaustive_grid(torch, H, W, u, method):
    # the FP32 pass only chooses which points the double-float evaluation visits: records
    # must be byte-identical to evaluating the whole grid in double-float. Extra frames: the
    # reference itself (peak at offset 0), a noise-free frame shifted by half a grid step
    # (two points tie in exact arithmetic) and a flat frame (every point ties: more
    # candidates than the list holds, so the kernel falls back to the whole grid)
    ref, frames = pairs(H, W, 16, seed=H + W + u, u16=False)
    half = synth.gaussian_spot(H, W, H / 2 + 0.5 / u, W / 2 - 0.5 / u, 2.5, 1500.0, 10.0)
    extra = np.array([ref, half, np.full((H, W), 7.0)], np.float32)
    frames = np.concatenate([frames, extra])
    recs = []
    for exhaustive in (False, True):
        t = C.Tracker(ref, upsample=u, method=method, in_dtype="f32", max_batch=64, exhaustive=exhaustive)
        recs.append(track(torch, t, frames))
        t.close()
    assert recs[0].tobytes() == recs[1].tobytes()
    check(ref, frames[:16], recs[0][:16], u, method)


def test_non_finite_frame_is_flagged(torch):
    ref, frames = pairs(40, 40, 3, seed=9, u16=False)
    frames[1, 7, 9] = np.nan
    t = tracker(ref, 50, oracle.CC_U, False)
    res = track(torch, t, frames)
    t.close()
    assert res[1]["flags"] & C.R_NONFINITE and res[1]["flags"] & C.R_GENERIC
    assert not (res[0]["flags"] & C.R_NONFINITE) and not (res[2]["flags"] & C.R_NONFINITE)
    check(ref, frames[[0, 2]], res[[0, 2]], 50, oracle.CC_U)


def test_autotune_keeps_parity_and_batch_identity(torch):
    # a context of 96 x 96 with references of 48, 30 and 97 (prime: a single DFT level
    # is one of the candidates) added for ROI batches
    ref, frames = pairs(96, 96, 6, seed=11, u16=True)
    t = tracker(ref, 100, oracle.CC_U, True)
    extra = [pairs(N, N, 6, seed=12 + N, u16=True) for N in (48, 30, 97)]
    ids = [0] + [C.ccst_add_reference(t.ctx, r, *r.shape) for r, _ in extra]
    tuned = C.ccst_autotune(t.ctx, reps=2)
    assert len(tuned) == 4 and {(x["H"], x["W"]) for x in tuned} == {(96, 96), (48, 48), (30, 30), (97, 97)}
    for x in tuned:
        assert x["H"] % x["H1"] == 0 and x["W"] % x["W1"] == 0 and x["threads"] in (256, 512)
        assert x["us_per_frame"] > 0 and x["timed"] > 0
    sets = [(ref, frames)] + extra
    devs = [dev(torch, f) for _, f in sets]
    rois = [d[i] for d in devs for i in range(6)]
    rid = [ids[k] for k in range(4) for _ in range(6)]
    batch = C.make_rois(rois, rid)
    assert len(C.ccst_autotune(t.ctx, 2, batch, len(rois))) == 4          # tuned on this batch
    out = t.empty_results(len(rois))
    C.ccst_track_rois(t.ctx, batch, len(rois), out)
    C.ccst_sync(t.ctx)
    mixed = C.decode(out)
    res = track(torch, t, frames)
    check(ref, frames, res, 100, oracle.CC_U)
    assert mixed[:6].tobytes() == res.tobytes()                  # ROI path = tracking path
    for k, (r, f) in enumerate(extra, start=1):
        check(r, f, mixed[6 * k:6 * (k + 1)], 100, oracle.CC_U)
    t.close()
