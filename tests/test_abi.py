"""The C-ABI library loads on a CPU-only machine and exports every entry point the header declares."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2310_08770_b300 import ccst as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    with open(os.path.join(ROOT, "include", "ccst.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ccst_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_08770_b300 import build
    build.build()
    return C.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    # and the binding wraps each one under the same name
    wrapped = {n for n, _, _ in C._SIGS}
    assert set(names) <= wrapped


def test_version_and_defaults(lib):
    assert C.ccst_version() == 10000
    p = C.ccst_default_params()
    assert (p.upsample, p.method, p.eps, p.in_dtype, p.max_batch, p.flags) == (100, 0, 200.0, 0, 256, 1)


def test_result_record_layout():
    assert C.RESULT_DTYPE.itemsize == 24
    assert C.ccst_params.stream.offset == 32 and ctypes.sizeof(C.ccst_params) == 48


def test_invalid_arguments_return_codes_without_gpu(lib):
    ctx = ctypes.c_void_p()
    ref = np.zeros((64, 64), np.float32)
    # null ref / null out
    assert lib.ccst_create(None, 64, 64, None, ctypes.byref(ctx)) == C.E_INVALID
    assert lib.ccst_create(ref.ctypes.data, 64, 64, None, None) == C.E_INVALID
    # shapes outside [8, 256] are rejected before touching the device
    for H, W in [(0, 64), (4, 4), (64, 300), (257, 64), (7, 100)]:
        assert lib.ccst_create(ref.ctypes.data, H, W, None, ctypes.byref(ctx)) == C.E_SHAPE
    p = C.ccst_default_params()
    p.upsample = 0
    assert lib.ccst_create(ref.ctypes.data, 64, 64, ctypes.byref(p), ctypes.byref(ctx)) == C.E_INVALID
    p = C.ccst_default_params()
    p.method = 7
    assert lib.ccst_create(ref.ctypes.data, 64, 64, ctypes.byref(p), ctypes.byref(ctx)) == C.E_INVALID
    assert b"method" in lib.ccst_last_error(None)
    # calls on a NULL context
    assert lib.ccst_track(None, None, 0, 0, None) == C.E_INVALID
    assert lib.ccst_sync(None) == C.E_INVALID
    assert lib.ccst_grid_size(None) == C.E_INVALID
    lib.ccst_destroy(None)           # NULL-safe


def test_python_binding_raises_cleanly_without_device(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(C.CcstError):
        C.ccst_create(np.zeros((64, 64), np.float32), 64, 64)


def test_new_record_layouts_match_the_header():
    # ccst_roi: {const void* frame; int32 H, W; int64 pitch_elems; int32 ref_id, reserved}
    assert ctypes.sizeof(C.ccst_roi) == 32
    assert (C.ccst_roi.frame.offset, C.ccst_roi.H.offset, C.ccst_roi.W.offset, C.ccst_roi.pitch_elems.offset,
            C.ccst_roi.ref_id.offset) == (0, 8, 12, 16, 24)
    # ccst_server_stats: 4 x uint64, 4 x double, 4 x int64
    assert ctypes.sizeof(C.ccst_server_stats_t) == 96 and C.ccst_server_stats_t.in_flight.offset == 64
    assert C.ccst_server_stats_t.budget_bytes.offset == 88
    # ccst_server_config: 2 x int32, int64, uint32, int32
    assert ctypes.sizeof(C.ccst_server_config) == 24 and C.ccst_server_config.budget_bytes.offset == 8
    # ccst_tune_result: 6 x int32, double
    assert ctypes.sizeof(C.ccst_tune_result) == 32 and C.ccst_tune_result.us_per_frame.offset == 24


def test_null_handles_are_rejected_without_gpu(lib):
    n = None
    assert lib.ccst_rt_begin(n, n, 0, 0.1, 0.9) == C.E_INVALID
    assert lib.ccst_rt_track(n, n, 1, 0, n) == C.E_INVALID
    assert lib.ccst_set_reference_frame(n, n, 0) == C.E_INVALID
    assert lib.ccst_offline_update(n, n, 1, 0, n) == C.E_INVALID
    assert lib.ccst_offline_track(n, n, 1, 0, 1, n) == C.E_INVALID
    assert lib.ccst_reference_status(n, n) == C.E_INVALID
    assert lib.ccst_peak_continuous(n, n, 1, 0, n, n, n) == C.E_INVALID
    assert lib.ccst_backward(n, n, 1, 0, n, n, n, n) == C.E_INVALID
    assert lib.ccst_drift_correct(n, 5, 0.1, 0.9, 0.0, 100, n, n) == C.E_INVALID
    assert lib.ccst_drift_correct(n, -1, 0.1, 0.9, 0.0, 100, n, n) == C.E_INVALID
    rid = ctypes.c_int()
    assert lib.ccst_add_reference(n, n, 32, 32, ctypes.byref(rid)) == C.E_INVALID
    assert lib.ccst_track_rois(n, n, 1, n) == C.E_INVALID
    out = ctypes.c_void_p()
    assert lib.ccst_server_create(n, 4, 4, ctypes.byref(out)) == C.E_INVALID
    cfg = C.ccst_server_config(16, 2, 1 << 20, 0, 0)
    assert lib.ccst_server_create_ex(n, ctypes.byref(cfg), ctypes.byref(out)) == C.E_INVALID
    assert lib.ccst_set_reference_image(n, n) == C.E_INVALID
    assert lib.ccst_refine_reference(n, n, 4, 0, n, 2, 0.01, n, n) == C.E_INVALID
    i64 = ctypes.c_int64()
    assert lib.ccst_graph_stats(n, ctypes.byref(i64), ctypes.byref(i64), ctypes.byref(i64)) == C.E_INVALID
    assert lib.ccst_fp32_fma_peak(n, 100, n, n) == C.E_INVALID
    assert lib.ccst_server_submit(n, 0, n, 0, n) == C.E_INVALID
    done = ctypes.c_int()
    assert lib.ccst_server_poll(n, 1, 0, n, ctypes.byref(done)) == C.E_INVALID
    st = C.ccst_server_stats_t()
    assert lib.ccst_server_read_stats(n, 0, ctypes.byref(st)) == C.E_INVALID
    lib.ccst_server_destroy(n)
    assert lib.ccst_debug_rt_timeout(n, n, 0, n) == C.E_INVALID
    assert lib.ccst_autotune(n, 3, n, 0, n, 0, n) == C.E_INVALID
    assert lib.ccst_debug_reference(n, n) == C.E_INVALID
