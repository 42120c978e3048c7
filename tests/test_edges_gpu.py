"""Edge cases of the reference-update, adjoint and serving entry points: padded row pitch
gives the records of unpadded frames bit for bit, a frame set as the reference tracks as
the oracle does against it, and the server takes float32 frames."""
import numpy as np
import pytest

import oracle
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


def frames_of(n, N, seed, u16):
    rng = np.random.default_rng(seed)
    d = rng.uniform(-2, 2, size=(n, 2))
    f = np.array([rng.poisson(synth.gaussian_spot(N, N, N / 2 + p[0], N / 2 + p[1], 2.5, 900.0, 15.0)) for p in d])
    return f.astype(np.uint16) if u16 else f.astype(np.float32)


def dev(torch, a, pad=0):
    if pad:
        buf = np.zeros(a.shape[:-1] + (a.shape[-1] + pad,), a.dtype)
        buf[..., :a.shape[-1]] = a
        a = buf
    t = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda()
    return t.view(torch.uint16) if a.dtype == np.uint16 else t


@pytest.mark.parametrize("u16", [True, False])
def test_padded_pitch_real_time_and_offline(torch, u16):
    fr = frames_of(10, 32, seed=1, u16=u16)
    el = "u16" if u16 else "f32"
    recs = []
    for pad in (0, 8):
        d = dev(torch, fr, pad)
        pitch = 32 + pad if pad else 0
        t = C.Tracker(np.zeros((32, 32), np.float32), upsample=50, in_dtype=el, max_batch=16)
        rt = t.empty_results(9)
        C.ccst_rt_begin(t.ctx, d[0], pitch, 0.2, 0.8)
        C.ccst_rt_track(t.ctx, d[1:], 9, pitch, rt)
        off = t.empty_results(10)
        C.ccst_offline_track(t.ctx, d, 10, pitch, 2, off)
        C.ccst_sync(t.ctx)
        recs.append((C.decode(rt).tobytes(), C.decode(off).tobytes()))
        t.close()
    assert recs[0] == recs[1]


def test_padded_pitch_adjoint(torch):
    fr = frames_of(6, 64, seed=2, u16=False)
    ref = synth.gaussian_spot(64, 64, 32, 32, 2.5, 900.0, 15.0).astype(np.float32)
    outs = []
    for pad in (0, 4):
        d = dev(torch, fr, pad)
        pitch = 64 + pad if pad else 0
        t = C.Tracker(ref, upsample=100, in_dtype="f32", max_batch=8)
        rec = t.empty_results(6)
        C.ccst_track(t.ctx, d, 6, pitch, rec)
        peak = torch.empty((6, 2), dtype=torch.float64, device="cuda")
        gI = torch.empty((6, 64, 64), dtype=torch.float32, device="cuda")
        gE = torch.empty((64, 64), dtype=torch.float32, device="cuda")
        g = torch.ones((6, 2), dtype=torch.float32, device="cuda")
        C.ccst_peak_continuous(t.ctx, d, 6, pitch, rec, peak, None)
        C.ccst_backward(t.ctx, d, 6, pitch, rec, g, gI, gE)
        C.ccst_sync(t.ctx)
        outs.append((peak.cpu().numpy().tobytes(), gI.cpu().numpy().tobytes(), gE.cpu().numpy().tobytes()))
        t.close()
    assert outs[0] == outs[1]


@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_frame_set_as_reference_tracks_like_the_oracle(torch, method):
    fr = frames_of(12, 64, seed=3, u16=True)
    t = C.Tracker(np.ones((64, 64), np.float32), upsample=100, method=method, in_dtype="u16", max_batch=16)
    d = dev(torch, fr)
    C.ccst_set_reference_frame(t.ctx, d[0])
    out = t.empty_results(11)
    C.ccst_track(t.ctx, d[1:], 11, 0, out)
    C.ccst_sync(t.ctx)
    res = C.decode(out)
    t.close()
    want = oracle.track_batch(fr[1:].astype(np.float64), fr[0].astype(np.float64), u=100, method=method)
    for g, o in zip(res, want):
        assert ((g["ipy"], g["ipx"]) == (o["ipy"], o["ipx"]) or o["int_margin"] < 1e-12)
        assert (abs(g["dx"] - o["dx32"]) <= 1e-3 and abs(g["dy"] - o["dy32"]) <= 1e-3) or o["sub_margin"] < 1e-12


def test_server_with_float32_frames(torch):
    fr = frames_of(8, 64, seed=4, u16=False)
    ref = synth.gaussian_spot(64, 64, 32, 32, 2.5, 900.0, 15.0).astype(np.float32)
    t = C.Tracker(ref, upsample=100, in_dtype="f32", max_batch=8)
    out = t.empty_results(8)
    C.ccst_track(t.ctx, dev(torch, fr), 8, 0, out)
    C.ccst_sync(t.ctx)
    want = C.decode(out)
    srv = C.ccst_server_create(t.ctx, 16, 16)
    try:
        tickets = [C.ccst_server_submit(srv, 0, fr[i]) for i in range(8)]
        got = [C.ccst_server_poll(srv, tk, 5_000_000) for tk in tickets]
    finally:
        C.ccst_server_destroy(srv)
        t.close()
    assert all(g.tobytes() == w.tobytes() for g, w in zip(got, want))


def test_track_tensor_is_a_view_of_the_records(torch):
    fr = frames_of(300, 32, seed=6, u16=True)
    ref = synth.gaussian_spot(32, 32, 16, 16, 2.5, 900.0, 15.0).astype(np.float32)
    t = C.Tracker(ref, upsample=100, in_dtype="u16", max_batch=128)
    d = dev(torch, fr)
    rec = t.track(d)
    ten = t.track_tensor(d)
    torch.cuda.synchronize()
    t.close()
    assert ten.shape == (300, 3) and ten.dtype == torch.float32 and ten.is_cuda
    got = ten.cpu().numpy()
    assert np.array_equal(got[:, 0], rec["dx"]) and np.array_equal(got[:, 1], rec["dy"])
    assert np.array_equal(got[:, 2], rec["peak"])
