"""The allocation-free entry point gives the same results as the context-based one.

ccst_track_static serves callers that may not allocate device memory once they are
running (for example a camera loop that reserved all GPU memory at start-up, or a
plug-in whose host owns the memory pool). It keeps everything a context would own
in one fixed device array that every call shares. This test calls it twice in a row
with different shapes, methods and upsampling factors -- so the second call runs
over the first call's leftovers -- and compares each result with ccst_create +
ccst_track on the same frames, under the parity tests' tolerance. It lives in a file
of its own that pytest collects last.
"""
import numpy as np
import pytest

from paper_2310_08770_b300 import ccst as C
from paper_2310_08770_b300 import synth

pytestmark = pytest.mark.gpu

TOL_PX = 1e-3


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08770_b300 import build
    build.build()
    return _t


def _context_results(torch, ref, frames_dev, n, params, H, W):
    ctx = C.ccst_create(ref, H, W, params)
    out = torch.empty((n, 24), dtype=torch.uint8, device="cuda")
    C.ccst_track(ctx, frames_dev, n, 0, out)
    C.ccst_sync(ctx)
    C.ccst_destroy(ctx)
    return C.decode(out)


def _static_results(torch, ref, frames_dev, n, params, H, W):
    ref_dev = torch.from_numpy(np.ascontiguousarray(ref, np.float32)).cuda()
    out = torch.empty((n, 24), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    C.ccst_track_static(ref_dev, H, W, params, frames_dev, n, 0, out)
    torch.cuda.synchronize()
    return C.decode(out)


def _same(a, b):
    assert np.array_equal(a["ipy"], b["ipy"]) and np.array_equal(a["ipx"], b["ipx"])
    assert np.max(np.abs(a["dx"] - b["dx"])) <= TOL_PX and np.max(np.abs(a["dy"] - b["dy"])) <= TOL_PX
    assert np.allclose(a["peak"], b["peak"], rtol=2e-5, atol=0)


def test_static_entry_matches_context_entry_twice_in_a_row(torch):
    # call 1: the frame-stream workload (uint16 128x128, u = 100, CC-U)
    s = synth.frame_stream(seed=11, n=96)
    f1 = torch.from_numpy(s.frames.view(np.int16)).cuda().view(torch.uint16)
    p1 = C.ccst_default_params()
    p1.max_batch = 96
    r1_static = _static_results(torch, s.ref, f1, 96, p1, 128, 128)
    r1_ctx = _context_results(torch, s.ref, f1, 96, p1, 128, 128)
    _same(r1_static, r1_ctx)

    # call 2, straight after: another shape, method, upsampling and element type
    rng = np.random.default_rng(3)
    H, W = 64, 32
    ref2 = synth.gaussian_spot(H, W, 32.0, 16.0, 2.5, 900.0, 15.0).astype(np.float32)
    fr2 = np.array([rng.poisson(synth.gaussian_spot(H, W, 32 + d[1], 16 + d[0], 2.5, 900.0, 15.0))
                    for d in rng.uniform(-4, 4, size=(40, 2))], np.float32)
    f2 = torch.from_numpy(fr2).cuda()
    p2 = C.ccst_default_params()
    p2.upsample, p2.method, p2.in_dtype, p2.eps, p2.max_batch = 37, C.CC_SN, C.F32, 200.0, 40
    r2_static = _static_results(torch, ref2, f2, 40, p2, H, W)
    r2_ctx = _context_results(torch, ref2, f2, 40, p2, H, W)
    _same(r2_static, r2_ctx)


def test_static_entry_rejects_oversized_requests(torch):
    ref = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
    p = C.ccst_default_params()
    p.upsample = 2048                        # upsampling tables alone exceed the fixed array
    out = torch.empty((1, 24), dtype=torch.uint8, device="cuda")
    frames = torch.zeros((1, 128, 128), dtype=torch.float32, device="cuda")
    with pytest.raises(C.CcstError) as e:
        C.ccst_track_static(ref, 128, 128, p, frames, 1, 0, out)
    assert e.value.code == C.E_SHAPE and "2 MiB" in str(e.value)
    with pytest.raises(C.CcstError) as e:
        C.ccst_track_static(ref, 256, 256, None, frames, 1, 0, out)
    assert e.value.code == C.E_SHAPE
    p = C.ccst_default_params()
    p.method = C.CC_SN
    p.eps = float("nan")                     # ccst_create refuses the same parameters
    with pytest.raises(C.CcstError) as e:
        C.ccst_track_static(ref, 128, 128, p, frames, 1, 0, out)
    assert e.value.code == C.E_INVALID
