"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar: integer peaks identical; |dx|, |dy| within 1e-3 px of the oracle's float32
result (with u = 100 the grid step is 0.01 px, so this means the same grid
point). The only exception allowed is a genuine tie: a frame whose oracle top-2
margin (relative to sum|X|/HW) is below 1e-12, where both choices are maxima
to float64 precision. ``peak`` agrees to 2e-5 relative.
"""
import ctypes
import json
import os

import numpy as np
import pytest

import oracle
from paper_2310_08770_b300 import ccst as C
from paper_2310_08770_b300 import synth

pytestmark = pytest.mark.gpu

TOL_PX = 1e-3
TIE = 1e-12
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08770_b300 import build
    build.build()
    return _t


def run_gpu(torch, ref, frames, u=100, method=0, eps=200.0, graphs=False, debug=False, pitch_pad=0,
            max_batch=256):
    torch.cuda.synchronize()
    stream = torch.cuda.Stream() if graphs else None
    frames = np.asarray(frames)
    in_dtype = "u16" if frames.dtype == np.uint16 else "f32"
    if in_dtype == "f32":
        frames = frames.astype(np.float32)
    n, H, W = frames.shape
    t = C.Tracker(ref.astype(np.float32), upsample=u, method=method, eps=eps, in_dtype=in_dtype,
                  max_batch=max_batch, graphs=graphs, stream=stream)
    tdt = torch.uint16 if in_dtype == "u16" else torch.float32
    if pitch_pad:
        host = np.zeros((n, H, W + pitch_pad), dtype=frames.dtype)
        host[:, :, :W] = frames
        dev = torch.from_numpy(host.view(np.int16) if in_dtype == "u16" else host).cuda()
        pitch = W + pitch_pad
    else:
        dev = torch.from_numpy(frames.view(np.int16) if in_dtype == "u16" else frames).cuda()
        pitch = 0
    dev = dev.view(tdt) if in_dtype == "u16" else dev
    out = torch.empty((n, 24), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    surf_i = surf_s = None
    if debug:
        surf_i = torch.empty((n, H, W), dtype=torch.float32, device="cuda")
        surf_s = torch.empty((n, t.M, t.M), dtype=torch.float32, device="cuda")
        C.ccst_debug_surfaces(t.ctx, dev, n, pitch, out, surf_i, surf_s)
    else:
        for s in range(0, n, max_batch):
            e = min(n, s + max_batch)
            C.ccst_track(t.ctx, dev[s:e], e - s, pitch, out[s:e])
    C.ccst_sync(t.ctx)
    res = C.decode(out)
    t.close()
    if debug:
        return res, surf_i.cpu().numpy(), surf_s.cpu().numpy()
    return res


def compare(res, orc, label=""):
    bad = []
    for i, (g, o) in enumerate(zip(res, orc)):
        int_ok = (g["ipy"], g["ipx"]) == (o["ipy"], o["ipx"]) or o["int_margin"] < TIE
        sub_ok = (abs(float(g["dx"]) - o["dx32"]) <= TOL_PX and abs(float(g["dy"]) - o["dy32"]) <= TOL_PX) \
            or o["sub_margin"] < TIE or o["int_margin"] < TIE
        peak_ok = abs(float(g["peak"]) - o["peak"]) <= 2e-5 * max(abs(o["peak"]), o["scale"] * 1e-3)
        if not (int_ok and sub_ok and peak_ok):
            bad.append((i, (float(g["dx"]), float(g["dy"]), int(g["ipy"]), int(g["ipx"]), float(g["peak"]),
                            int(g["flags"])),
                        (o["dx"], o["dy"], o["ipy"], o["ipx"], o["peak"], o["sub_margin"])))
    assert not bad, f"{label}: {len(bad)} of {len(orc)} frames differ; first: {bad[:5]}"


def flag_counts(res):
    f = res["flags"]
    return {name: int(np.sum((f & bit) != 0)) for name, bit in
            (("int", C.R_INT_GUARD), ("sub", C.R_SUB_GUARD), ("df64", C.R_DF64), ("overflow", C.R_OVERFLOW))}


# ------------------------------------------------------------------ single pair
@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_single_pair(torch, method):
    p = synth.single_pair(seed=0)
    res = run_gpu(torch, p.ref, p.frame[None], u=100, method=method)
    orc = [oracle.track_one(p.frame, p.ref, u=100, method=method)]
    compare(res, orc, "single pair")
    with open(os.path.join(GOLDEN, "single_pair_oracle.json")) as f:
        gold = json.load(f)["ccu" if method == 0 else "ccsn"]
    assert float(res["dx"][0]) == np.float32(gold["dx"]) and float(res["dy"][0]) == np.float32(gold["dy"])


# ------------------------------------------------------------------ exact cases
@pytest.mark.parametrize("N,sigma,u", [(64, 3.0, 100), (128, 2.5, 100), (64, 3.0, 256), (32, 2.0, 37)])
def test_noise_free_subpixel_exact(torch, N, sigma, u):
    rng = np.random.default_rng(1)
    c = N / 2.0
    ref = synth.gaussian_spot(N, N, c, c, sigma, 1000.0, 10.0)
    frames, expect = [], []
    while len(frames) < 24:
        d = rng.uniform(-4, 4, size=2)
        if min(abs((u * d[0]) % 1 - 0.5), abs((u * d[1]) % 1 - 0.5)) < 0.1:
            continue
        frames.append(synth.gaussian_spot(N, N, c + d[1], c + d[0], sigma, 1000.0, 10.0))
        expect.append((round(u * d[0]) / u, round(u * d[1]) / u))
    res = run_gpu(torch, ref, np.array(frames, np.float32), u=u)
    for r, (ex, ey) in zip(res, expect):
        assert float(r["dx"]) == np.float32(ex) and float(r["dy"]) == np.float32(ey)


@pytest.mark.parametrize("shape", [(64, 64), (128, 128), (32, 64), (128, 16), (8, 8)])
def test_integer_rolls_exact(torch, shape):
    rng = np.random.default_rng(4)
    H, W = shape
    ref = synth.random_texture(rng, H, W)
    shifts = [(0, 0), (1, -2), (H // 2, -(W // 2) + 1), (-(H // 2) + 1, W // 2), (H // 4, W // 3)]
    frames = np.array([np.roll(ref, s, axis=(0, 1)) for s in shifts], np.float32)
    for method in (oracle.CC_U, oracle.CC_SN):
        res = run_gpu(torch, ref, frames, u=100, method=method)
        for r, (dy, dx) in zip(res, shifts):
            assert (int(r["ipy"]), int(r["ipx"])) == (dy, dx)
            if method == oracle.CC_U:
                assert float(r["dx"]) == dx and float(r["dy"]) == dy


# ------------------------------------------------------------------ frame stream
def test_frame_stream_first_batch(torch):
    s = synth.frame_stream(seed=0, n=10_000, count=256)
    res = run_gpu(torch, s.ref, s.frames, u=100)
    orc = oracle.track_batch_parallel(s.frames, s.ref, u=100)
    compare(res, orc, "stream batch 0")
    # the estimates track the known trajectory
    err = np.hypot(res["dx"] - s.d_true[:, 0], res["dy"] - s.d_true[:, 1])
    assert np.median(err) < 0.05
    print("flags", flag_counts(res))


def test_frame_stream_full_size_sampled(torch):
    """The full 10,000-frame stream in 256-frame graph batches; a sample checked frame by frame."""
    s = synth.frame_stream(seed=0, n=10_000)
    res = run_gpu(torch, s.ref, s.frames, u=100, graphs=True)
    assert res.shape == (10_000,)
    # properties that hold at every frame: inside the refinement square, near the truth
    assert np.all(np.abs(res["dx"] - res["ipx"]) <= 0.76) and np.all(np.abs(res["dy"] - res["ipy"]) <= 0.76)
    err = np.hypot(res["dx"] - s.d_true[:, 0], res["dy"] - s.d_true[:, 1])
    assert np.max(err) < 0.5 and np.median(err) < 0.05
    assert not np.any(res["flags"] & (C.R_OVERFLOW | C.R_NONFINITE))
    rng = np.random.default_rng(123)
    idx = np.sort(rng.choice(10_000, size=160, replace=False))
    idx = np.unique(np.concatenate([idx, [0, 255, 256, 9_983, 9_984, 9_999]]))
    orc = oracle.track_batch_parallel(s.frames[idx], s.ref, u=100)
    compare(res[idx], orc, "stream sample")
    # every frame the guard had to re-decide is checked too
    gidx = np.nonzero(res["flags"] & (C.R_SUB_GUARD | C.R_DF64 | C.R_INT_GUARD))[0][:200]
    if len(gidx):
        compare(res[gidx], oracle.track_batch_parallel(s.frames[gidx], s.ref, u=100), "guarded frames")
    print("flags over 10000 frames", flag_counts(res))


# ------------------------------------------------------------------ shapes, u, methods
# (128, 128, 120): the refinement grid no longer fits one chunk, stages A/B run in chunks;
# (128, 128, 200): the stage tables no longer fit shared memory, the plain-FP32 stages read
# them from global memory
@pytest.mark.parametrize("H,W,u", [(8, 8, 7), (16, 16, 1), (16, 32, 2), (32, 32, 37), (64, 32, 100),
                                   (32, 128, 100), (128, 64, 50), (64, 64, 256), (128, 128, 11),
                                   (128, 128, 120), (128, 128, 200), (32, 8, 50), (64, 8, 100),
                                   (128, 8, 100)])
@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_shapes_and_upsampling(torch, H, W, u, method):
    rng = np.random.default_rng(H * 1000 + W + u)
    ref = synth.gaussian_spot(H, W, H / 2, W / 2, max(1.2, min(H, W) / 16), 800.0, 12.0)
    frames = []
    for _ in range(12):
        d = rng.uniform(-min(H, W) / 6, min(H, W) / 6, size=2)
        frames.append(rng.poisson(synth.gaussian_spot(H, W, H / 2 + d[1], W / 2 + d[0],
                                                      max(1.2, min(H, W) / 16), 800.0, 12.0)))
    frames = np.array(frames, np.float32)
    res = run_gpu(torch, ref, frames, u=u, method=method)
    orc = oracle.track_batch(frames, ref, u=u, method=method)
    compare(res, orc, f"{H}x{W} u={u} m={method}")


# every shape the power-of-two kernel accepts (H, W in {8, ..., 128}): each one is its own
# instantiation, with its own choice of stage forms
@pytest.mark.parametrize("H", [8, 16, 32, 64, 128])
@pytest.mark.parametrize("W", [8, 16, 32, 64, 128])
@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_every_power_of_two_shape(torch, H, W, method):
    rng = np.random.default_rng(7 * H + W)
    sigma = max(1.2, min(H, W) / 16)
    ref = synth.gaussian_spot(H, W, H / 2, W / 2, sigma, 800.0, 12.0)
    d = rng.uniform(-min(H, W) / 6, min(H, W) / 6, size=(6, 2))
    frames = np.array([rng.poisson(synth.gaussian_spot(H, W, H / 2 + p[1], W / 2 + p[0], sigma, 800.0, 12.0))
                       for p in d], np.float32)
    res = run_gpu(torch, ref, frames, u=40, method=method)
    orc = oracle.track_batch(frames, ref, u=40, method=method)
    compare(res, orc, f"{H}x{W} m={method}")


# uint16 input, aligned (16-byte vector loads) and with a row pitch of W + 3 (scalar loads),
# on the narrow and the square shapes: the same records either way, and the oracle's
@pytest.mark.parametrize("H,W", [(8, 8), (128, 8), (8, 128), (64, 64), (128, 128)])
def test_uint16_ingest_aligned_and_pitched(torch, H, W):
    rng = np.random.default_rng(11 * H + W)
    sigma = max(1.2, min(H, W) / 16)
    ref = synth.gaussian_spot(H, W, H / 2, W / 2, sigma, 800.0, 12.0)
    d = rng.uniform(-min(H, W) / 6, min(H, W) / 6, size=(6, 2))
    frames = np.array([rng.poisson(synth.gaussian_spot(H, W, H / 2 + p[1], W / 2 + p[0], sigma, 800.0, 12.0))
                       for p in d]).astype(np.uint16)
    a = run_gpu(torch, ref, frames, u=50)
    b = run_gpu(torch, ref, frames, u=50, pitch_pad=3)
    assert a.tobytes() == b.tobytes()
    compare(a, oracle.track_batch(frames.astype(np.float64), ref, u=50), f"{H}x{W} u16")


# the upsampling factor across the plan's switch points (the tcgen05 contraction at 128^2,
# the chunked stages, the stage tables in shared or in global memory, odd and even grids)
U_SWEEP = [1, 2, 3, 4, 5, 8, 13, 16, 33, 64, 101, 127, 150, 181, 255, 301, 512]


@pytest.mark.parametrize("N", [64, 128])
@pytest.mark.parametrize("u", U_SWEEP)
def test_upsampling_factor_sweep(torch, N, u):
    rng = np.random.default_rng(N + 13 * u)
    ref = synth.gaussian_spot(N, N, N / 2, N / 2, 2.5, 1000.0, 10.0)
    d = rng.uniform(-3, 3, size=(6, 2))
    frames = np.array([rng.poisson(synth.gaussian_spot(N, N, N / 2 + p[1], N / 2 + p[0], 2.5, 1000.0, 10.0))
                       for p in d], np.float32)
    methods = (oracle.CC_U, oracle.CC_SN) if N == 128 and u in (1, 64, 101, 255, 512) else (oracle.CC_U,)
    for method in methods:
        res = run_gpu(torch, ref, frames, u=u, method=method)
        orc = oracle.track_batch(frames, ref, u=u, method=method)
        compare(res, orc, f"{N}x{N} u={u} m={method}")


def test_ccsn_stream_batch(torch):
    s = synth.frame_stream(seed=3, n=128, H=64, W=64, sigma=3.0, amplitude=1000.0, background=10.0, step=0.5,
                           bound=10.0)
    res = run_gpu(torch, s.ref, s.frames, u=100, method=oracle.CC_SN, eps=200.0)
    orc = oracle.track_batch_parallel(s.frames, s.ref, u=100, method=oracle.CC_SN, eps=200.0)
    compare(res, orc, "cc-sn stream")


def test_textures_ragged_batch(torch):
    rng = np.random.default_rng(8)
    ref = synth.random_texture(rng, 64, 64)
    frames = []
    for _ in range(37):                         # ragged: not a multiple of anything
        d = rng.uniform(-8, 8, size=2)
        mu = np.real(np.fft.ifft2(np.fft.fft2(ref) * np.exp(
            -2j * np.pi * (np.fft.fftfreq(64)[:, None] * d[1] + np.fft.fftfreq(64)[None, :] * d[0]))))
        frames.append(rng.poisson(np.maximum(mu, 0)))
    frames = np.array(frames, np.float32)
    res = run_gpu(torch, ref, frames, u=100, max_batch=16)
    compare(res, oracle.track_batch(frames, ref, u=100), "textures")


# ------------------------------------------------------------------ guard levels
@pytest.mark.parametrize("delta", [1e-4, 3e-5, 2e-5, 1.2e-5, 1e-5, 3e-6, 1e-6, 1e-7])
def test_near_half_bin_shifts_exercise_guard(torch, delta):
    """Noise-free spots placed delta px past a half-bin: top-2 margins shrink with delta
    (about 1e-3 * delta relative), walking the decision through every guard level."""
    N, sigma, u = 64, 3.0, 100
    rng = np.random.default_rng(int(1 / delta))
    ref = synth.gaussian_spot(N, N, 32.0, 32.0, sigma, 1000.0, 10.0)
    frames = []
    for _ in range(16):
        k = rng.integers(-150, 150, size=2)
        d = (k + 0.5) / u + delta * rng.choice([-1, 1], size=2)
        frames.append(synth.gaussian_spot(N, N, 32.0 + d[1], 32.0 + d[0], sigma, 1000.0, 10.0))
    frames = np.array(frames, np.float32)
    res = run_gpu(torch, ref, frames, u=u)
    orc = oracle.track_batch(frames, ref, u=u)
    compare(res, orc, f"half-bin delta={delta}")
    print("delta", delta, flag_counts(res))


# ------------------------------------------------------------------ FP32 error vs thresholds
def test_fp32_surface_error_is_far_below_guard_thresholds(torch):
    """The guard is only sound if its thresholds bound the FP32 surface error. Measure the
    error of the FP32 delta surface near its maximum against the FP64 oracle."""
    s = synth.frame_stream(seed=5, n=64)
    res, si, ss = run_gpu(torch, s.ref, s.frames, u=100, debug=True)
    eps32 = 2.0 ** -23
    worst_sub, worst_int = 0.0, 0.0
    for f in range(len(s.frames)):
        a, b, sense = oracle.surface_operands(s.frames[f], s.ref)
        X = oracle.product_spectrum(a, b)
        H, W = a.shape
        scale = float(np.sum(np.abs(X.real) + np.abs(X.imag)))     # sum w|X| over the full plane
        c64 = np.real(np.fft.ifft2(X)) * H * W
        worst_int = max(worst_int, np.max(np.abs(si[f] - c64)) / scale)
        py, px = int(res["ipy"][f]), int(res["ipx"][f])
        cu = oracle.upsampled_cc(X, py, px, 100) * H * W
        M = cu.shape[0]
        d64 = cu - cu[M // 2, M // 2]
        near = d64 >= d64.max() - 1e-5 * scale
        worst_sub = max(worst_sub, np.max(np.abs(ss[f] - d64)[near]) / scale)
    print(f"worst FP32 errors / (eps32 * sum|X|): integer {worst_int / eps32:.3g}, sub-pixel {worst_sub / eps32:.3g}")
    assert worst_sub < 0.125 * 1.0 * eps32      # tau0 = 1 eps32: keep an 8x margin
    assert worst_int < 0.125 * 32.0 * eps32     # tau_int = 32 eps32


# ------------------------------------------------------------------ paths and edges
def test_host_path_graphs_and_submit_match_device_path(torch):
    s = synth.frame_stream(seed=2, n=300, count=300)
    base = run_gpu(torch, s.ref, s.frames[:256], u=100)
    stream = torch.cuda.Stream()
    t = C.Tracker(s.ref, upsample=100, graphs=True, stream=stream, profile=True)
    host = t.track_host(s.frames[:256])
    assert np.array_equal(host, base)
    dev = torch.from_numpy(s.frames.view(np.int16)).cuda().view(torch.uint16)
    out = torch.empty((256, 24), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    for _ in range(3):                       # capture once, replay twice
        C.ccst_track(t.ctx, dev[:256], 256, 0, out)
    C.ccst_sync(t.ctx)
    assert np.array_equal(C.decode(out), base)
    ms, launches = C.ccst_profile_kernel_ms(t.ctx)
    assert launches >= 1 and ms > 0
    out2 = torch.empty((256, 24), dtype=torch.uint8, device="cuda")
    tk = C.ccst_submit(t.ctx, dev[:256], 256, out2)
    done = False
    for _ in range(10000):
        if C.ccst_poll(t.ctx, tk, 1000):
            done = True
            break
    assert done and np.array_equal(C.decode(out2), base)
    with pytest.raises(C.CcstError):
        C.ccst_poll(t.ctx, tk, 0)            # released ticket is unknown now
    t.close()


def test_pipelined_host_path_matches_device_path(torch):
    """ccst_submit_host: six batches (two full rounds of its staging slots, a ragged last
    one) with three in flight; every batch's results equal the device path's."""
    s = synth.frame_stream(seed=4, n=1400, count=1400)
    sizes = [256, 256, 100, 256, 256, 200]
    starts = np.cumsum([0] + sizes[:-1])
    base = run_gpu(torch, s.ref, s.frames, u=100)
    t = C.Tracker(s.ref, upsample=100)
    pinned = torch.from_numpy(s.frames.view(np.int16)).pin_memory().numpy().view(np.uint16)
    outs = [torch.empty((256 * 24,), dtype=torch.uint8).pin_memory().numpy().view(C.RESULT_DTYPE)
            for _ in sizes]
    pending = []
    for k, (lo, n) in enumerate(zip(starts, sizes)):
        pending.append((k, C.ccst_submit_host(t.ctx, pinned[lo:lo + n], n, 0, outs[k])))
        if len(pending) == 3:
            k0, tk = pending.pop(0)
            while not C.ccst_poll(t.ctx, tk, 100000):
                pass
    for k0, tk in pending:
        while not C.ccst_poll(t.ctx, tk, 100000):
            pass
    for k, (lo, n) in enumerate(zip(starts, sizes)):
        assert np.array_equal(outs[k][:n], base[lo:lo + n]), f"batch {k}"
    t.close()


def test_bounded_table_wait_reports_timeout_and_context_survives(torch):
    """With the table copies withheld, every CTA's bounded wait runs out: each frame it
    reached reports CCST_R_TIMEOUT, nothing faults, and the context still tracks."""
    s = synth.frame_stream(seed=5, n=64, count=16)
    base = run_gpu(torch, s.ref, s.frames, u=100)
    t = C.Tracker(s.ref, upsample=100, max_batch=16)
    dev = torch.from_numpy(s.frames.view(np.int16)).cuda().view(torch.uint16)
    out = torch.zeros((16, 24), dtype=torch.uint8, device="cuda")
    C.ccst_debug_timeout(t.ctx, dev, 16, 0, out)
    C.ccst_sync(t.ctx)
    res = C.decode(out)
    assert np.all(res["flags"] & C.R_TIMEOUT), res["flags"]
    out2 = torch.zeros((16, 24), dtype=torch.uint8, device="cuda")
    C.ccst_track(t.ctx, dev, 16, 0, out2)
    C.ccst_sync(t.ctx)
    assert np.array_equal(C.decode(out2), base)
    t.close()


def test_edge_cases(torch):
    H = W = 32
    ref = synth.gaussian_spot(H, W, 16.0, 16.0, 2.0, 500.0, 5.0).astype(np.float32)
    t = C.Tracker(ref, upsample=10, in_dtype="f32", max_batch=8)
    out = torch.empty((8, 24), dtype=torch.uint8, device="cuda")
    frames = torch.zeros((9, H, W), dtype=torch.float32, device="cuda")
    C.ccst_track(t.ctx, frames, 0, 0, out)                       # n = 0: no-op
    with pytest.raises(C.CcstError) as e:
        C.ccst_track(t.ctx, frames, 9, 0, out)                   # n > max_batch
    assert e.value.code == C.E_INVALID
    with pytest.raises(C.CcstError):
        C.ccst_track(t.ctx, frames, 1, W - 1, out)               # pitch < W
    with pytest.raises(C.CcstError) as e:
        C.ccst_backward(t.ctx, frames, 1, 0, out, None, None, None)     # no upstream gradient
    assert e.value.code == C.E_INVALID
    # constant frame: every point ties; lowest index everywhere, as in the oracle
    frames[0] = 7.0
    C.ccst_track(t.ctx, frames, 1, 0, out)
    C.ccst_sync(t.ctx)
    r = C.decode(out)[0]
    o = oracle.track_one(np.full((H, W), 7.0), ref, u=10)
    assert (int(r["ipy"]), int(r["ipx"]), float(r["dx"]), float(r["dy"])) == (o["ipy"], o["ipx"], o["dx32"], o["dy32"])
    t.close()
    # row pitch larger than W
    s = synth.frame_stream(seed=4, n=20, H=64, W=64, sigma=3.0, amplitude=1000.0, background=10.0)
    a = run_gpu(torch, s.ref, s.frames, u=100, pitch_pad=24)
    b = run_gpu(torch, s.ref, s.frames, u=100)
    assert np.array_equal(a, b)
    # a frame with zero pixels under CC-SN
    f = s.frames[:2].copy()
    f[:, :10, :] = 0
    compare(run_gpu(torch, s.ref, f, method=oracle.CC_SN), oracle.track_batch(f, s.ref, method=oracle.CC_SN),
            "zeros cc-sn")


def test_pair_difference_error_is_far_below_tau1(torch):
    """Calibrates the middle guard level: the FP32 pair difference v(jb) - v(ja) between the
    winner and its neighbours, against the oracle's exact FP64 difference. Also reports the
    error left by the FP32 product spectrum alone (FP64 accumulation over it)."""
    s = synth.frame_stream(seed=7, n=64)
    frames = s.frames
    res = run_gpu(torch, s.ref, frames, u=100)
    M, h0, u = 150, 75, 100
    n = len(frames)
    eps32 = 2.0 ** -23
    worst32 = worst64 = 0.0
    dev = torch.from_numpy(frames.view(np.int16)).cuda().view(torch.uint16)
    t = C.Tracker(s.ref, upsample=u, max_batch=n)
    cus, scales = [], []
    for f in range(n):
        a, b, _ = oracle.surface_operands(frames[f], s.ref)
        X = oracle.product_spectrum(a, b)
        cus.append(oracle.upsampled_cc(X, int(res["ipy"][f]), int(res["ipx"][f]), u) * 128 * 128)
        scales.append(float(np.sum(np.abs(X.real) + np.abs(X.imag))))
    for dy, dx in [(0, 1), (1, 0), (1, 1), (0, -1), (-1, 0), (-1, 1), (2, 0), (0, 3)]:
        pairs = np.zeros((n, 2), np.int32)
        for f in range(n):
            jy = int(round(float(res["dy"][f]) * u)) - int(res["ipy"][f]) * u + h0
            jx = int(round(float(res["dx"][f]) * u)) - int(res["ipx"][f]) * u + h0
            jby, jbx = min(max(jy + dy, 0), M - 1), min(max(jx + dx, 0), M - 1)
            pairs[f] = (jy * M + jx, jby * M + jbx)
        pd = torch.from_numpy(pairs).cuda()
        d32 = torch.empty(n, dtype=torch.float32, device="cuda")
        d64 = torch.empty(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        C.ccst_debug_pairs(t.ctx, dev, n, 0, pd, d32, d64)
        C.ccst_sync(t.ctx)
        d32, d64 = d32.cpu().numpy(), d64.cpu().numpy()
        for f in range(n):
            cu = cus[f].ravel()
            exact = cu[pairs[f, 1]] - cu[pairs[f, 0]]
            worst32 = max(worst32, abs(d32[f] - exact) / scales[f])
            worst64 = max(worst64, abs(d64[f] - exact) / scales[f])
    t.close()
    print(f"pair-difference error / (eps32 sum|X|): FP32 guard {worst32 / eps32:.3g}, "
          f"FP64 over the FP32 spectrum {worst64 / eps32:.3g}")
    assert worst32 < 0.05 * eps32 / 8          # tau1 = 0.05 eps32 with an 8x margin


@pytest.mark.parametrize("graphs", [False, True])
def test_batches_in_flight_on_several_streams_match_one_at_a_time(torch, graphs):
    # The 10,000-frame stream as 40 batches (39 x 256 + 16) over three rotating streams, two
    # passes, into outputs pre-filled with a 0xFF sentinel: every record must be written and
    # byte-equal to the records of the same batches run one at a time on one stream. With
    # graphs, each (stream, batch) pair is captured exactly once: 40 instantiations, 80 replays.
    s = synth.frame_stream(seed=0, n=10_000)
    n = len(s.frames)
    dev = torch.from_numpy(s.frames.view(np.int16)).cuda().view(torch.uint16)
    bounds = [(lo, min(n, lo + 256)) for lo in range(0, n, 256)]
    assert len(bounds) == 40
    one_t = C.Tracker(s.ref, upsample=100, in_dtype="u16", max_batch=256)
    one = torch.full((n, 24), 0xFF, dtype=torch.uint8, device="cuda")
    for lo, hi in bounds:
        C.ccst_track(one_t.ctx, dev[lo:hi], hi - lo, 0, one[lo:hi])
    C.ccst_sync(one_t.ctx)
    one_t.close()
    streams = [torch.cuda.Stream() for _ in range(3)]
    t = C.Tracker(s.ref, upsample=100, in_dtype="u16", max_batch=256, graphs=graphs, stream=streams[0])
    for rep in range(2):
        many = torch.full((n, 24), 0xFF, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        for b, (lo, hi) in enumerate(bounds):
            C.ccst_set_stream(t.ctx, streams[b % 3].cuda_stream)
            C.ccst_track(t.ctx, dev[lo:hi], hi - lo, 0, many[lo:hi])
        torch.cuda.synchronize()
        got = many.cpu().numpy()
        unwritten = np.flatnonzero((got == 0xFF).all(axis=1))
        assert unwritten.size == 0, unwritten[:20]
        bad = np.flatnonzero((got != one.cpu().numpy()).any(axis=1))
        assert bad.size == 0, bad[:20]
        del many
    st = C.ccst_graph_stats(t.ctx)
    if graphs:
        assert st == {"instantiations": 40, "replays": 80, "cached": 40}, st
    else:
        assert st == {"instantiations": 0, "replays": 0, "cached": 0}, st
    t.close()
