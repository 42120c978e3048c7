"""The FP32 general-size kernel (square sides 48, 96, 192 and 256; mixed-radix (2, 3) FFTs,
one to four CTAs per frame). Its records must meet the FP64 oracle's parity bar (integer
peaks equal, |dx|, |dy| within 1e-3 px, genuine ties excepted); its surface and pair-
difference errors must sit far below the guard thresholds that certify its decisions; and
the frames it cannot certify (exact ties) must come back from the double-float kernel with
that kernel's own records."""
import numpy as np
import pytest

import oracle
from paper_2310_08770_b300 import ccst as C
from paper_2310_08770_b300 import synth

pytestmark = pytest.mark.gpu

TOL_PX = 1e-3
TIE = 1e-12
EPS32 = 2.0 ** -23
GEN = C.R_GENERIC | C.R_FP32_GENERAL
# guard thresholds of the FP32 general-size kernel, in eps32 * sum w|X| (CC-U, CC-SN)
TAU0 = {oracle.CC_U: {48: 1.0, 96: 1.0, 192: 1.0, 256: 1.0}, oracle.CC_SN: {48: 0.125, 96: 0.125, 192: 0.06, 256: 0.03}}
TAU1 = {oracle.CC_U: 0.02, oracle.CC_SN: 0.005}
TAU_INT = 32.0


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08770_b300 import build
    build.build()
    return _t


def spots(N, n, seed, u16=True, shift=3.0):
    """Noise-free spot reference at the centre; Poisson frames shifted U(-shift, shift) px."""
    rng = np.random.default_rng(seed)
    sigma, amp, bg = rng.uniform(1.8, 3.5), rng.uniform(400, 4000), rng.uniform(5, 40)
    ref = synth.gaussian_spot(N, N, N / 2, N / 2, sigma, amp, bg)
    d = rng.uniform(-shift, shift, size=(n, 2))
    fr = np.array([rng.poisson(synth.gaussian_spot(N, N, N / 2 + p[0], N / 2 + p[1], sigma, amp, bg)) for p in d])
    return ref.astype(np.float32), fr.astype(np.uint16 if u16 else np.float32)


def dev(torch, a, pad=0):
    if pad:
        buf = np.zeros(a.shape[:-1] + (a.shape[-1] + pad,), a.dtype)
        buf[..., :a.shape[-1]] = a
        a = buf
    t = torch.from_numpy(np.ascontiguousarray(a).view(np.int16) if a.dtype == np.uint16 else np.ascontiguousarray(a))
    t = t.cuda()
    return t.view(torch.uint16) if a.dtype == np.uint16 else t


def track(torch, ref, frames, u=100, method=0, exhaustive=False, pad=0):
    t = C.Tracker(ref, upsample=u, method=method, in_dtype="u16" if frames.dtype == np.uint16 else "f32",
                  max_batch=len(frames), exhaustive=exhaustive)
    d = dev(torch, frames, pad)
    out = t.empty_results(len(frames))
    C.ccst_track(t.ctx, d, len(frames), frames.shape[-1] + pad if pad else 0, out)
    C.ccst_sync(t.ctx)
    res = C.decode(out)
    t.close()
    return res


def check(ref, frames, res, u, method):
    bad = []
    for i, (f, g) in enumerate(zip(frames, res)):
        assert g["flags"] & GEN, (i, g["flags"])
        o = oracle.track_one(f.astype(np.float64), ref.astype(np.float64), u, method)
        int_ok = (g["ipy"], g["ipx"]) == (o["ipy"], o["ipx"]) or o["int_margin"] < TIE
        sub_ok = (abs(g["dx"] - o["dx32"]) <= TOL_PX and abs(g["dy"] - o["dy32"]) <= TOL_PX) or o["sub_margin"] < TIE
        if not (int_ok and sub_ok):
            bad.append((i, (g["ipy"], g["ipx"], g["dx"], g["dy"], g["flags"]), (o["ipy"], o["ipx"], o["dx32"], o["dy32"])))
        assert abs(g["peak"] - o["peak"]) <= 1e-5 * abs(o["peak"]), (i, g["peak"], o["peak"])
    assert not bad, bad


@pytest.mark.parametrize("N", [48, 96, 192, 256])
@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_sides_and_methods_match_the_oracle(torch, N, method):
    n = 16 if N <= 96 else 8
    ref, frames = spots(N, n, seed=40 + N + method, u16=(N + method) % 2 == 0)
    res = track(torch, ref, frames, 100, method)
    check(ref, frames, res, 100, method)
    fp32 = int(np.sum((res["flags"] & C.R_FP32_GENERAL) != 0))
    # CC-U frames of Poisson spots are certified by the FP32 levels (the rare fallback aside)
    if method == oracle.CC_U:
        assert fp32 >= n - 1, res["flags"]


@pytest.mark.parametrize("N,u", [(96, 1), (96, 3), (48, 37), (96, 120), (192, 256), (256, 256), (96, 300)])
def test_upsampling_factors(torch, N, u):
    # u = 256 at 256 x 256 splits the contraction into several t chunks; above u = 256 the
    # side has no FP32 plan and the double-float kernel alone tracks it
    ref, frames = spots(N, 6, seed=N + u, u16=True)
    res = track(torch, ref, frames, u, oracle.CC_U)
    check(ref, frames, res, u, oracle.CC_U)
    if u > 256:
        assert np.all((res["flags"] & C.R_FP32_GENERAL) == 0)
    else:
        assert np.sum((res["flags"] & C.R_FP32_GENERAL) != 0) >= 5


@pytest.mark.parametrize("N", [48, 96, 192, 256])
@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_fp32_surface_errors_are_far_below_the_thresholds(torch, N, method):
    """The FP32 integer surface and the peak-relative upsampled surface (near its extremum)
    against the FP64 oracle, in eps32 * sum w|X|: an 8x margin below tau_int and tau0."""
    n, M = 8, 150
    ref, frames = spots(N, n, seed=60 + N + method)
    t = C.Tracker(ref, upsample=100, method=method, in_dtype="u16", max_batch=n)
    d = dev(torch, frames)
    out = t.empty_results(n)
    si = torch.full((n, N, N), float("nan"), device="cuda")
    ss = torch.full((n, M, M), float("nan"), device="cuda")
    C.ccst_debug_surfaces(t.ctx, d, n, 0, out, si, ss)
    C.ccst_sync(t.ctx)
    res = C.decode(out)
    t.close()
    si, ss = si.cpu().numpy(), ss.cpu().numpy()
    worst_i = worst_s = 0.0
    seen = 0
    for f in range(n):
        a, b, sense = oracle.surface_operands(frames[f].astype(np.float64), ref.astype(np.float64), method)
        X = oracle.product_spectrum(a, b)
        scale = float(np.sum(np.abs(X.real) + np.abs(X.imag)))
        c64 = np.real(oracle.idft2(X)) * N * N
        if not np.all(np.isfinite(si[f])):
            continue
        seen += 1
        worst_i = max(worst_i, float(np.max(np.abs(si[f] - c64))) / scale)
        py, px = int(res["ipy"][f]), int(res["ipx"][f])
        cu = oracle.upsampled_cc(X, py, px, 100) * N * N
        d64 = cu - cu[M // 2, M // 2]
        if np.all(np.isfinite(ss[f])):
            near = sense * d64 >= (sense * d64).max() - 1e-5 * scale
            worst_s = max(worst_s, float(np.max(np.abs(ss[f] - d64)[near])) / scale)
    print(f"N={N} method={method}: worst FP32 errors / (eps32 sum|X|): integer {worst_i / EPS32:.3g}, "
          f"sub-pixel {worst_s / EPS32:.3g}")
    assert seen >= n - 1
    assert worst_i < TAU_INT * EPS32 / 8
    assert worst_s < TAU0[method][N] * EPS32 / 8


@pytest.mark.parametrize("N", [48, 192])
@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_pair_difference_error_is_far_below_tau1(torch, N, method):
    """v(jb) - v(ja) by the FP32 pair-difference level, for the oracle's winner ja and grid
    neighbours jb, against the oracle's FP64 difference: an 8x margin below tau1."""
    n, M, u = 12, 150, 100
    ref, frames = spots(N, n, seed=80 + N + method)
    orcs, cus, scales = [], [], []
    for f in range(n):
        a, b, _ = oracle.surface_operands(frames[f].astype(np.float64), ref.astype(np.float64), method)
        X = oracle.product_spectrum(a, b)
        o = oracle.track_one(frames[f].astype(np.float64), ref.astype(np.float64), u, method)
        orcs.append(o)
        cus.append((oracle.upsampled_cc(X, o["ipy"], o["ipx"], u) * N * N).ravel())
        scales.append(float(np.sum(np.abs(X.real) + np.abs(X.imag))))
    t = C.Tracker(ref, upsample=u, method=method, in_dtype="u16", max_batch=n)
    d = dev(torch, frames)
    worst = 0.0
    done = 0
    for dy, dx in [(0, 1), (1, 0), (1, 1), (0, -1), (-1, 0), (-2, 1), (0, 3)]:
        pairs = np.zeros((n, 2), np.int32)
        for f, o in enumerate(orcs):
            jby, jbx = min(max(o["jy"] + dy, 0), M - 1), min(max(o["jx"] + dx, 0), M - 1)
            pairs[f] = (o["jy"] * M + o["jx"], jby * M + jbx)
        pd = torch.from_numpy(pairs).cuda()
        d32 = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        d64 = torch.empty(n, dtype=torch.float64, device="cuda")
        C.ccst_debug_pairs(t.ctx, d, n, 0, pd, d32, d64)
        C.ccst_sync(t.ctx)
        d32 = d32.cpu().numpy()
        for f in range(n):
            if np.isfinite(d32[f]):
                exact = cus[f][pairs[f, 1]] - cus[f][pairs[f, 0]]
                worst = max(worst, abs(float(d32[f]) - exact) / scales[f])
                done += 1
    t.close()
    print(f"N={N} method={method}: pair-difference error / (eps32 sum|X|) {worst / EPS32:.3g}")
    assert done >= 6 * n
    assert worst < TAU1[method] * EPS32 / 8


@pytest.mark.parametrize("N", [96, 256])
def test_ties_fall_back_to_the_double_float_kernel(torch, N):
    # a flat frame (every shift ties), the reference itself and a noise-free frame shifted by
    # half a grid step (two grid points tie exactly) beside ordinary frames: the frames the
    # FP32 levels cannot certify carry CCST_R_GENERIC and are byte-identical to the double-
    # float kernel's records; the others decide as that kernel does
    u = 50
    ref, frames = spots(N, 6, seed=90 + N, u16=False)
    half = synth.gaussian_spot(N, N, N / 2 + 0.5 / u, N / 2 - 0.5 / u, 2.5, 1500.0, 10.0)
    frames = np.concatenate([frames, np.array([np.full((N, N), 7.0), ref, half], np.float32)])
    fast = track(torch, ref, frames, u)
    slow = track(torch, ref, frames, u, exhaustive=True)
    assert fast[6]["flags"] & C.R_GENERIC and not fast[6]["flags"] & C.R_FP32_GENERAL
    for i in range(len(frames)):
        if fast[i]["flags"] & C.R_GENERIC:
            assert fast[i].tobytes() == slow[i].tobytes(), i
        else:
            assert fast[i]["flags"] & C.R_FP32_GENERAL
            for k in ("ipy", "ipx", "dx", "dy"):
                assert fast[i][k] == slow[i][k], (i, k)
            assert abs(fast[i]["peak"] - slow[i]["peak"]) <= 1e-5 * abs(slow[i]["peak"])
    check(ref, frames[:6], fast[:6], u, oracle.CC_U)


@pytest.mark.parametrize("N,method", [(96, oracle.CC_U), (48, oracle.CC_SN), (192, oracle.CC_U)])
def test_decisions_equal_the_double_float_kernel(torch, N, method):
    ref, frames = spots(N, 24 if N < 192 else 10, seed=110 + N + method, u16=True)
    fast = track(torch, ref, frames, 100, method)
    slow = track(torch, ref, frames, 100, method, exhaustive=True)
    for i in range(len(frames)):
        for k in ("ipy", "ipx", "dx", "dy"):
            assert fast[i][k] == slow[i][k], (i, k, fast[i], slow[i])
        assert abs(fast[i]["peak"] - slow[i]["peak"]) <= 1e-5 * abs(slow[i]["peak"])


@pytest.mark.parametrize("N", [48, 192])
def test_padded_rows_and_float_frames(torch, N):
    # rows `pad` elements apart take the scalar loads instead of 16-byte vectors: same records
    ref, frames = spots(N, 6, seed=130 + N, u16=False)
    plain = track(torch, ref, frames)
    padded = track(torch, ref, frames, pad=3)
    assert plain.tobytes() == padded.tobytes()
    check(ref, frames, plain, 100, oracle.CC_U)


def test_rois_of_every_fp32_side_graph_and_direct(torch):
    # one work list with all four FP32 sides and power-of-two sides: direct and graph-
    # captured replays give the same records, which meet the oracle
    rng = np.random.default_rng(140)
    sides = [256, 48, 64, 192, 96, 128, 48, 96, 32, 256]
    items = []
    for N in sides:
        ref, fr = spots(N, 1, seed=int(rng.integers(1 << 30)))
        items.append((ref, fr[0]))
    frames = [dev(torch, f) for _, f in items]
    ref0 = synth.gaussian_spot(32, 32, 16, 16, 2.0, 500.0, 10.0).astype(np.float32)
    recs = []
    for graphs in (False, True):
        st = torch.cuda.Stream() if graphs else None
        t = C.Tracker(ref0, upsample=100, in_dtype="u16", graphs=graphs, stream=st)
        ids = [C.ccst_add_reference(t.ctx, r, *r.shape) for r, _ in items]
        rois = C.make_rois(frames, ids)
        for _ in range(2 if graphs else 1):
            out = t.empty_results(len(items))
            C.ccst_track_rois(t.ctx, rois, len(items), out)
            C.ccst_sync(t.ctx)
            recs.append(C.decode(out).tobytes())
        t.close()
    assert recs[0] == recs[1] == recs[2]
    res = np.frombuffer(recs[0], C.RESULT_DTYPE)
    for (ref, f), g, N in zip(items, res, sides):
        if N in (48, 96, 192, 256):
            check(ref, f[None], g[None], 100, oracle.CC_U)


def test_fallbacks_of_both_chained_fp32_launches_reach_the_double_float_kernel(torch):
    # flat ROIs (every shift ties) at 96 and 48 px, whose FP32 launches run one behind the
    # other on the second stream, beside power-of-two ROIs on the first: the double-float
    # kernel, launched after the join, must find the fallbacks of both launches. Every ROI's
    # record equals the one its own context gives for that frame alone (direct and graph-
    # replayed calls alike).
    rng = np.random.default_rng(150)
    sides = [96, 128, 48, 32, 96, 48, 64, 128, 96, 48]
    flat = {4, 5}
    items = []
    for i, N in enumerate(sides):
        ref, fr = spots(N, 1, seed=int(rng.integers(1 << 30)))
        items.append((ref, np.full((N, N), 7, np.uint16) if i in flat else fr[0]))
    alone = [track(torch, ref, f[None], 100)[0] for ref, f in items]
    for i in flat:
        assert alone[i]["flags"] & C.R_GENERIC and not alone[i]["flags"] & C.R_FP32_GENERAL, (i, alone[i])
    frames = [dev(torch, f) for _, f in items]
    ref0 = synth.gaussian_spot(32, 32, 16, 16, 2.0, 500.0, 10.0).astype(np.float32)
    for graphs in (False, True):
        st = torch.cuda.Stream() if graphs else None
        t = C.Tracker(ref0, upsample=100, in_dtype="u16", graphs=graphs, stream=st)
        ids = [C.ccst_add_reference(t.ctx, r, *r.shape) for r, _ in items]
        rois = C.make_rois(frames, ids)
        for _ in range(2 if graphs else 1):
            out = t.empty_results(len(items))
            C.ccst_track_rois(t.ctx, rois, len(items), out)
            C.ccst_sync(t.ctx)
            res = C.decode(out)
            for i in range(len(items)):
                assert res[i].tobytes() == alone[i].tobytes(), (graphs, i, sides[i], res[i], alone[i])
        t.close()


@pytest.mark.parametrize("N", [48, 96])
@pytest.mark.parametrize("u", [2, 5, 16, 45, 64, 101, 181])
def test_upsampling_factor_sweep(torch, N, u):
    # the plan's chunking (one chunk, or 40-row chunks beside the shared-memory stage-B
    # table at 96 px from h0 >= 32) across u
    ref, frames = spots(N, 6, seed=160 + N + u)
    res = track(torch, ref, frames, u)
    check(ref, frames, res, u, oracle.CC_U)


@pytest.mark.parametrize("N", [48, 96, 192, 256])
def test_integer_near_ties_are_decided_in_double_float(torch, N):
    # noise-free spots shifted by 1/2 + d px along x: the integer shifts 0 and 1 nearly tie
    # (d = 1e-4 .. 1e-6 px, far inside the FP32 threshold), and the kernel re-decides them
    # from its double-float spectrum (CCST_R_INT_GUARD); an exact half-pixel shift of a
    # symmetric spot ties exactly and goes to the double-float kernel
    ref = synth.gaussian_spot(N, N, N / 2, N / 2, 2.5, 2000.0, 10.0).astype(np.float32)
    ds = [1e-4, -1e-4, 3e-5, 1e-5, -3e-6, 1e-6]
    frames = np.array([synth.gaussian_spot(N, N, N / 2 + 0.3, N / 2 + 0.5 + d, 2.5, 2000.0, 10.0) for d in ds],
                      np.float32)
    res = track(torch, ref, frames, 100)
    guarded = int(np.sum((res["flags"] & C.R_INT_GUARD) != 0))
    assert guarded >= 3, res["flags"]
    check(ref, frames, res, 100, oracle.CC_U)


@pytest.mark.parametrize("H,W", [(256, 128), (128, 256)])
@pytest.mark.parametrize("method", [oracle.CC_U, oracle.CC_SN])
def test_table_one_shape_both_ways(torch, H, W, method):
    # the paper's Table I frame shape, 256 x 128, and its transpose: clusters of two CTAs
    rng = np.random.default_rng(150 + H + method)
    ref = synth.gaussian_spot(H, W, H / 2, W / 2, 3.0, 1500.0, 15.0).astype(np.float32)
    d = rng.uniform(-3, 3, size=(8, 2))
    frames = np.array([rng.poisson(synth.gaussian_spot(H, W, H / 2 + p[0], W / 2 + p[1], 3.0, 1500.0, 15.0))
                       for p in d]).astype(np.uint16)
    res = track(torch, ref, frames, 100, method)
    check(ref, frames, res, 100, method)
    if method == oracle.CC_U:
        assert np.sum((res["flags"] & C.R_FP32_GENERAL) != 0) >= 7, res["flags"]
