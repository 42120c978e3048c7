"""Thin ctypes binding of libccst (include/ccst.h).

Argument marshalling only: every step of the tracking path runs in the CUDA
library. torch is used for device memory and streams. The functions keep the C
names; :class:`Tracker` is a small convenience wrapper over them.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

CC_U = 0
CC_SN = 1
U16 = 0
F32 = 1
FLAG_TIE_GUARD = 0x1
FLAG_GRAPHS = 0x2
FLAG_PROFILE = 0x4
FLAG_EXHAUSTIVE = 0x8

R_INT_GUARD = 0x01
R_SUB_GUARD = 0x02
R_DF64 = 0x04
R_OVERFLOW = 0x08
R_NONFINITE = 0x10
R_TIMEOUT = 0x20
R_RT_STALE = 0x40
R_GENERIC = 0x80
R_FP32_GENERAL = 0x100

OK, E_INVALID, E_SHAPE, E_UNSUPPORTED, E_NOMEM, E_CUDA, E_TIMEOUT, E_BUSY = 0, -1, -2, -3, -4, -5, -6, -7
_CODES = {0: "OK", -1: "E_INVALID", -2: "E_SHAPE", -3: "E_UNSUPPORTED", -4: "E_NOMEM",
          -5: "E_CUDA", -6: "E_TIMEOUT", -7: "E_BUSY"}

RESULT_DTYPE = np.dtype([("dx", "<f4"), ("dy", "<f4"), ("peak", "<f4"),
                         ("ipy", "<i4"), ("ipx", "<i4"), ("flags", "<u4")])


class ccst_roi(ctypes.Structure):
    _fields_ = [("frame", ctypes.c_void_p), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("pitch_elems", ctypes.c_int64), ("ref_id", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ccst_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("mean_batch", ctypes.c_double), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("max_us", ctypes.c_double), ("in_flight", ctypes.c_int64),
                ("bytes_in_flight", ctypes.c_int64), ("max_bytes_in_flight", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64)]


class ccst_server_config(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("max_in_flight", ctypes.c_int32), ("budget_bytes", ctypes.c_int64),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32)]


class ccst_tune_result(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("H1", ctypes.c_int32), ("W1", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("timed", ctypes.c_int32), ("us_per_frame", ctypes.c_double)]


class ccst_params(ctypes.Structure):
    _fields_ = [("upsample", ctypes.c_int32), ("method", ctypes.c_int32), ("eps", ctypes.c_float),
                ("in_dtype", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("max_H", ctypes.c_int32),
                ("max_W", ctypes.c_int32), ("stream", ctypes.c_void_p), ("flags", ctypes.c_uint32)]


class CcstError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


_LIB = None


def library_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "libccst.so")


# (name, restype, argtypes) of every declared entry point
_SIGS = [
    ("ccst_version", ctypes.c_int, []),
    ("ccst_default_params", ctypes.c_int, [ctypes.POINTER(ccst_params)]),
    ("ccst_create", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ccst_params),
                                   ctypes.POINTER(ctypes.c_void_p)]),
    ("ccst_track", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_void_p]),
    ("ccst_track_host", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_void_p]),
    ("ccst_set_stream", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ccst_fp32_fma_peak", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]),
    ("ccst_graph_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    ("ccst_sync", ctypes.c_int, [ctypes.c_void_p]),
    ("ccst_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_uint64)]),
    ("ccst_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("ccst_submit_host", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    ("ccst_peak_continuous", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ccst_backward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ccst_set_reference_image", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ccst_refine_reference", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    ("ccst_destroy", None, [ctypes.c_void_p]),
    ("ccst_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("ccst_grid_size", ctypes.c_int, [ctypes.c_void_p]),
    ("ccst_profile_kernel_ms", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_int64)]),
    ("ccst_profile_reset", ctypes.c_int, [ctypes.c_void_p]),
    ("ccst_debug_surfaces", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ccst_add_reference", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]),
    ("ccst_track_rois", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ccst_roi), ctypes.c_int64, ctypes.c_void_p]),
    ("ccst_server_create", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    ("ccst_server_create_ex", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ccst_server_config),
                                             ctypes.POINTER(ctypes.c_void_p)]),
    ("ccst_server_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.POINTER(ctypes.c_uint64)]),
    ("ccst_server_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_int)]),
    ("ccst_server_read_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ccst_server_stats_t)]),
    ("ccst_server_loadgen", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_uint64,
                                           ctypes.POINTER(ccst_server_stats_t)]),
    ("ccst_server_destroy", None, [ctypes.c_void_p]),
    ("ccst_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.POINTER(ccst_tune_result), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("ccst_rt_begin", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                     ctypes.c_double]),
    ("ccst_rt_track", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_void_p]),
    ("ccst_drift_correct", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    ("ccst_set_reference_frame", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    ("ccst_offline_update", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_void_p]),
    ("ccst_offline_track", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int, ctypes.c_void_p]),
    ("ccst_reference_status", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    ("ccst_debug_reference", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ccst_debug_rt_timeout", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    ("ccst_debug_timeout", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_void_p]),
    ("ccst_debug_pairs", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ccst_track_static", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ccst_params),
                                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]),
    ("ccst_static_last_error", ctypes.c_char_p, []),
]


def lib() -> ctypes.CDLL:
    """Load libccst.so (once). Raises if the library has not been built."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise ImportError(f"libccst.so not found at {path}; build it with "
                              "`python -m paper_2310_08770_b300.build`")
        L = ctypes.CDLL(path)
        for name, res, args in _SIGS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(code, ctx=None):
    if code != OK:
        msg = lib().ccst_last_error(ctx)
        raise CcstError(code, msg.decode() if msg else "")
    return code


def _ptr(x):
    """Device or host address of a torch tensor or numpy array."""
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if x is None:
        return None
    return int(x)


# ---------------------------------------------------------------- C-named wrappers
def ccst_version() -> int:
    return lib().ccst_version()


def ccst_default_params() -> ccst_params:
    p = ccst_params()
    _check(lib().ccst_default_params(ctypes.byref(p)))
    return p


def ccst_create(ref, H: int, W: int, params: ccst_params | None = None) -> ctypes.c_void_p:
    """ref: float32 H x W (host numpy or CUDA tensor), copied by the library."""
    ctx = ctypes.c_void_p()
    p = ctypes.byref(params) if params is not None else None
    _check(lib().ccst_create(_ptr(ref), int(H), int(W), p, ctypes.byref(ctx)))
    return ctx


def ccst_track(ctx, frames_dev, n: int, pitch_elems: int, out_dev) -> None:
    _check(lib().ccst_track(ctx, _ptr(frames_dev), int(n), int(pitch_elems), _ptr(out_dev)), ctx)


def ccst_track_host(ctx, frames_host, n: int, pitch_elems: int, out_host) -> None:
    _check(lib().ccst_track_host(ctx, _ptr(frames_host), int(n), int(pitch_elems), _ptr(out_host)), ctx)


def ccst_set_stream(ctx, stream) -> None:
    _check(lib().ccst_set_stream(ctx, stream), ctx)


def ccst_graph_stats(ctx) -> dict:
    """Graph instantiations, replays and cached graphs of the context so far."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ccst_graph_stats(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), ctx)
    return {"instantiations": a.value, "replays": b.value, "cached": c.value}


def ccst_fp32_fma_peak(stream=None, iters: int = 20000) -> dict:
    """Measured and nominal FP32 FMA throughput of the current device, TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = lib().ccst_fp32_fma_peak(stream, int(iters), ctypes.byref(a), ctypes.byref(b))
    if rc:
        raise CcstError(rc, "ccst_fp32_fma_peak failed")
    return {"tflops": a.value, "nominal_tflops": b.value}


def ccst_sync(ctx) -> None:
    _check(lib().ccst_sync(ctx), ctx)


def ccst_submit(ctx, frames_dev, n: int, out_dev) -> int:
    t = ctypes.c_uint64()
    _check(lib().ccst_submit(ctx, _ptr(frames_dev), int(n), _ptr(out_dev), ctypes.byref(t)), ctx)
    return t.value


def ccst_submit_host(ctx, frames_host, n: int, pitch_elems: int, out_host) -> int:
    t = ctypes.c_uint64()
    _check(lib().ccst_submit_host(ctx, _ptr(frames_host), int(n), int(pitch_elems), _ptr(out_host),
                                  ctypes.byref(t)), ctx)
    return t.value


def ccst_poll(ctx, ticket: int, timeout_us: int) -> bool:
    done = ctypes.c_int()
    rc = lib().ccst_poll(ctx, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(done))
    if rc == E_TIMEOUT:
        return False
    _check(rc, ctx)
    return bool(done.value)


def ccst_add_reference(ctx, ref, H: int, W: int) -> int:
    """Add a reference (float32 H x W, numpy or torch, host or device) for ccst_track_rois."""
    if not hasattr(ref, "data_ptr"):
        ref = np.ascontiguousarray(ref, dtype=np.float32)
    rid = ctypes.c_int()
    _check(lib().ccst_add_reference(ctx, _ptr(ref), int(H), int(W), ctypes.byref(rid)), ctx)
    return rid.value


def make_rois(frames, ref_ids) -> ctypes.Array:
    """ccst_roi descriptors for a list of (H, W) CUDA tensors and their reference ids."""
    arr = (ccst_roi * len(frames))()
    for i, (f, r) in enumerate(zip(frames, ref_ids)):
        arr[i].frame = f.data_ptr()
        arr[i].H, arr[i].W = int(f.shape[-2]), int(f.shape[-1])
        arr[i].pitch_elems = int(f.stride(-2))
        arr[i].ref_id = int(r)
    return arr


def ccst_track_rois(ctx, rois, n, out_dev) -> None:
    _check(lib().ccst_track_rois(ctx, rois, int(n), _ptr(out_dev)), ctx)


def ccst_server_create(ctx, slots: int, max_batch: int):
    out = ctypes.c_void_p()
    _check(lib().ccst_server_create(ctx, int(slots), int(max_batch), ctypes.byref(out)), ctx)
    return out.value


def ccst_server_create_ex(ctx, max_batch: int, max_in_flight: int, budget_bytes: int):
    cfg = ccst_server_config(int(max_batch), int(max_in_flight), int(budget_bytes), 0, 0)
    out = ctypes.c_void_p()
    _check(lib().ccst_server_create_ex(ctx, ctypes.byref(cfg), ctypes.byref(out)), ctx)
    return out.value


def ccst_server_submit(srv, ref_id: int, frame_host, pitch_elems: int = 0, keep: bool = True):
    """Submit one host frame (numpy); returns the ticket (keep) or None. Raises CcstError
    (E_BUSY when the admission budget is full)."""
    t = ctypes.c_uint64()
    rc = lib().ccst_server_submit(srv, int(ref_id), _ptr(frame_host), int(pitch_elems),
                                  ctypes.byref(t) if keep else None)
    if rc != OK:
        raise CcstError(rc, "ccst_server_submit")
    return t.value if keep else None


def ccst_server_poll(srv, ticket: int, timeout_us: int):
    """The record (RESULT_DTYPE) of a finished ticket, or None on timeout."""
    rec = np.zeros(1, dtype=RESULT_DTYPE)
    done = ctypes.c_int()
    rc = lib().ccst_server_poll(srv, ctypes.c_uint64(ticket), int(timeout_us), rec.ctypes.data, ctypes.byref(done))
    if rc == E_TIMEOUT:
        return None
    if rc != OK:
        raise CcstError(rc, "ccst_server_poll")
    return rec[0]


def ccst_server_read_stats(srv, reset: bool = False) -> dict:
    st = ccst_server_stats_t()
    rc = lib().ccst_server_read_stats(srv, int(reset), ctypes.byref(st))
    if rc != OK:
        raise CcstError(rc, "ccst_server_read_stats")
    return {k: getattr(st, k) for k, _ in st._fields_}


def ccst_server_loadgen(srv, ref_ids, rates_hz, pools, seconds: float, seed: int = 0) -> dict:
    """Offered load from one host thread per camera; pools[k] is a contiguous numpy array
    (n_k, H_k, W_k) of camera k's frames in the context's dtype."""
    n = len(ref_ids)
    pools = [np.ascontiguousarray(p) for p in pools]
    st = ccst_server_stats_t()
    rc = lib().ccst_server_loadgen(srv, n, (ctypes.c_int * n)(*ref_ids), (ctypes.c_double * n)(*rates_hz),
                                   (ctypes.c_void_p * n)(*[p.ctypes.data for p in pools]),
                                   (ctypes.c_int * n)(*[p.shape[0] for p in pools]), float(seconds),
                                   ctypes.c_uint64(seed), ctypes.byref(st))
    if rc != OK:
        raise CcstError(rc, "ccst_server_loadgen")
    return {k: getattr(st, k) for k, _ in st._fields_}


def ccst_server_destroy(srv) -> None:
    if srv:
        lib().ccst_server_destroy(srv)


def ccst_rt_begin(ctx, frame0_dev, pitch_elems, a0, b1) -> None:
    _check(lib().ccst_rt_begin(ctx, _ptr(frame0_dev), int(pitch_elems), float(a0), float(b1)), ctx)


def ccst_rt_track(ctx, frames_dev, n, pitch_elems, out_dev) -> None:
    _check(lib().ccst_rt_track(ctx, _ptr(frames_dev), int(n), int(pitch_elems), _ptr(out_dev)), ctx)


def ccst_set_reference_frame(ctx, frame_dev, pitch_elems=0) -> None:
    _check(lib().ccst_set_reference_frame(ctx, _ptr(frame_dev), int(pitch_elems)), ctx)


def ccst_offline_update(ctx, frames_dev, n, pitch_elems, rec_dev) -> None:
    _check(lib().ccst_offline_update(ctx, _ptr(frames_dev), int(n), int(pitch_elems), _ptr(rec_dev)), ctx)


def ccst_offline_track(ctx, frames_dev, n, pitch_elems, passes, out_dev) -> None:
    _check(lib().ccst_offline_track(ctx, _ptr(frames_dev), int(n), int(pitch_elems), int(passes), _ptr(out_dev)),
           ctx)


def ccst_reference_status(ctx) -> bool:
    """True when a reference update gave up at a bounded wait (the reference is stale)."""
    st = ctypes.c_int()
    _check(lib().ccst_reference_status(ctx, ctypes.byref(st)), ctx)
    return bool(st.value)


def ccst_debug_reference(ctx, ref_dev) -> None:
    _check(lib().ccst_debug_reference(ctx, _ptr(ref_dev)), ctx)


def ccst_drift_correct(rec_dev, n, a0, b1, alpha, u, out_dev, stream=None) -> None:
    s = ctypes.c_void_p(0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream")
                                                  else int(stream)))
    rc = lib().ccst_drift_correct(_ptr(rec_dev), int(n), float(a0), float(b1), float(alpha), int(u),
                                  _ptr(out_dev), s)
    if rc != OK:
        raise CcstError(rc, "ccst_drift_correct failed")


def ccst_peak_continuous(ctx, frames_dev, n, pitch_elems, rec_dev, peak_dev, status_dev=None) -> None:
    _check(lib().ccst_peak_continuous(ctx, _ptr(frames_dev), int(n), int(pitch_elems), _ptr(rec_dev),
                                      _ptr(peak_dev), _ptr(status_dev)), ctx)


def ccst_backward(ctx, frames_dev, n, pitch_elems, rec_dev, g_dxdy_dev, g_frames_dev, g_ref_dev) -> None:
    _check(lib().ccst_backward(ctx, _ptr(frames_dev), int(n), int(pitch_elems), _ptr(rec_dev), _ptr(g_dxdy_dev),
                               _ptr(g_frames_dev), _ptr(g_ref_dev)), ctx)


def ccst_set_reference_image(ctx, image_dev) -> None:
    _check(lib().ccst_set_reference_image(ctx, _ptr(image_dev)), ctx)


def ccst_refine_reference(ctx, frames_dev, n, pitch_elems, target_dev, steps, step_rel, hist_dev,
                          ref_out_dev=None) -> None:
    _check(lib().ccst_refine_reference(ctx, _ptr(frames_dev), int(n), int(pitch_elems), _ptr(target_dev),
                                       int(steps), float(step_rel), _ptr(hist_dev), _ptr(ref_out_dev)), ctx)


def ccst_destroy(ctx) -> None:
    lib().ccst_destroy(ctx)


def ccst_autotune(ctx, reps: int = 3, rois=None, n_rois: int = 0) -> list:
    """Autotune the context's general-size plans (optionally on a ccst_roi batch from
    make_rois); one dict per plan (shape, splits, CTA size)."""
    arr = (ccst_tune_result * 64)()
    n = ctypes.c_int()
    _check(lib().ccst_autotune(ctx, int(reps), ctypes.cast(rois, ctypes.c_void_p) if rois is not None else None,
                               int(n_rois), arr, 64, ctypes.byref(n)), ctx)
    return [{k: getattr(arr[i], k) for k, _ in ccst_tune_result._fields_} for i in range(n.value)]


def ccst_grid_size(ctx) -> int:
    return _check_nonneg(lib().ccst_grid_size(ctx), ctx)


def ccst_profile_kernel_ms(ctx):
    """(total ms, launches) of the FP32 tracking kernel since the last reset."""
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    _check(lib().ccst_profile_kernel_ms(ctx, ctypes.byref(ms), ctypes.byref(cnt)), ctx)
    return ms.value, cnt.value


def ccst_profile_reset(ctx) -> None:
    _check(lib().ccst_profile_reset(ctx), ctx)


def _check_nonneg(v, ctx):
    if v < 0:
        _check(v, ctx)
    return v


def ccst_debug_surfaces(ctx, frames_dev, n, pitch_elems, out_dev, int_surf_dev, sub_surf_dev) -> None:
    _check(lib().ccst_debug_surfaces(ctx, _ptr(frames_dev), int(n), int(pitch_elems), _ptr(out_dev),
                                     _ptr(int_surf_dev), _ptr(sub_surf_dev)), ctx)


def ccst_debug_rt_timeout(ctx, frame_dev, pitch_elems, rec_dev) -> None:
    _check(lib().ccst_debug_rt_timeout(ctx, _ptr(frame_dev), int(pitch_elems), _ptr(rec_dev)), ctx)


def ccst_debug_timeout(ctx, frames_dev, n, pitch_elems, out_dev) -> None:
    _check(lib().ccst_debug_timeout(ctx, _ptr(frames_dev), int(n), int(pitch_elems), _ptr(out_dev)), ctx)


def ccst_debug_pairs(ctx, frames_dev, n, pitch_elems, pairs_dev, d32_dev, d64_dev) -> None:
    _check(lib().ccst_debug_pairs(ctx, _ptr(frames_dev), int(n), int(pitch_elems), _ptr(pairs_dev),
                                  _ptr(d32_dev), _ptr(d64_dev)), ctx)


def ccst_track_static(ref_dev, H: int, W: int, params: ccst_params | None, frames_dev, n: int,
                      pitch_elems: int, out_dev) -> None:
    """Allocation-free tracking: no context, all workspace in the library's fixed device array."""
    p = ctypes.byref(params) if params is not None else None
    rc = lib().ccst_track_static(_ptr(ref_dev), int(H), int(W), p, _ptr(frames_dev), int(n), int(pitch_elems),
                                 _ptr(out_dev))
    if rc != OK:
        raise CcstError(rc, lib().ccst_static_last_error().decode())


# ---------------------------------------------------------------- convenience wrapper
class Tracker:
    """One reference image, many frames.

    >>> t = Tracker(ref, upsample=100, method="ccu", in_dtype="u16")
    >>> res = t.track(frames)          # frames: CUDA tensor (n, H, W)
    >>> res["dx"], res["dy"]           # numpy structured array (RESULT_DTYPE)
    """

    def __init__(self, ref, upsample: int = 100, method: str | int = "ccu", eps: float = 200.0,
                 in_dtype: str | int = "u16", max_batch: int = 256, stream=None, graphs: bool = False,
                 tie_guard: bool = True, profile: bool = False, exhaustive: bool = False):
        import torch
        ref_np = ref.detach().cpu().numpy() if hasattr(ref, "detach") else np.asarray(ref)
        ref_np = np.ascontiguousarray(ref_np, dtype=np.float32)
        self.H, self.W = ref_np.shape
        p = ccst_default_params()
        p.upsample = int(upsample)
        p.method = {"ccu": CC_U, "ccsn": CC_SN}.get(method, method)
        p.eps = float(eps)
        p.in_dtype = {"u16": U16, "f32": F32}.get(in_dtype, in_dtype)
        p.max_batch = int(max_batch)
        if stream is None:
            stream = torch.cuda.current_stream()
        p.stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        p.flags = (FLAG_TIE_GUARD if tie_guard else 0) | (FLAG_GRAPHS if graphs else 0) | \
            (FLAG_PROFILE if profile else 0) | (FLAG_EXHAUSTIVE if exhaustive else 0)
        self.params = p
        self.max_batch = int(max_batch)
        self.ctx = ccst_create(ref_np, self.H, self.W, p)
        self.M = ccst_grid_size(self.ctx)
        self._torch = torch

    def close(self):
        if getattr(self, "ctx", None) is not None:
            ccst_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty_results(self, n: int):
        return self._torch.empty((n, 24), dtype=self._torch.uint8, device="cuda")

    def track_into(self, frames, out, pitch_elems: int = 0) -> None:
        """Asynchronous: frames (n, H, W) CUDA tensor, out (n, 24) uint8 CUDA tensor."""
        ccst_track(self.ctx, frames, frames.shape[0], pitch_elems, out)

    def track(self, frames) -> np.ndarray:
        """Synchronous convenience: all frames, in chunks of max_batch; returns RESULT_DTYPE records."""
        n = frames.shape[0]
        out = self.empty_results(n)
        for s in range(0, n, self.max_batch):
            e = min(n, s + self.max_batch)
            ccst_track(self.ctx, frames[s:e], e - s, 0, out[s:e])
        ccst_sync(self.ctx)
        return decode(out)

    def track_tensor(self, frames):
        """Device-side form: a float32 CUDA tensor (n, 3) of (dx, dy, peak), a view of the
        24-byte records (no host copy), valid once the context's stream has reached it."""
        n = frames.shape[0]
        out = self.empty_results(n)
        for s in range(0, n, self.max_batch):
            e = min(n, s + self.max_batch)
            ccst_track(self.ctx, frames[s:e], e - s, 0, out[s:e])
        return out.view(self._torch.float32)[:, :3]

    def rt_begin(self, frame0, a0: float, b1: float | None = None) -> None:
        """Start the real-time reference (Sec. III B) from frame0, a CUDA tensor (H, W)."""
        ccst_rt_begin(self.ctx, frame0, 0, a0, 1.0 - a0 if b1 is None else b1)

    def rt_track(self, frames) -> np.ndarray:
        """Real-time tracking of frames (n, H, W) CUDA tensor, one frame after another,
        the reference updated after each (Eq. (9)); returns RESULT_DTYPE records."""
        n = frames.shape[0]
        out = self.empty_results(n)
        ccst_rt_track(self.ctx, frames, n, 0, out)
        ccst_sync(self.ctx)
        return decode(out)

    def offline_track(self, frames, passes: int = 5) -> np.ndarray:
        """The offline method (Sec. III A) over frames (n, H, W) CUDA tensor: reference from
        frame 0, `passes` Eq. (8) updates; returns the records of the last pass."""
        n = frames.shape[0]
        out = self.empty_results(n)
        ccst_offline_track(self.ctx, frames, n, 0, passes, out)
        ccst_sync(self.ctx)
        return decode(out)

    def track_host(self, frames_np: np.ndarray) -> np.ndarray:
        n = frames_np.shape[0]
        frames_np = np.ascontiguousarray(frames_np)
        res = np.empty(n, dtype=RESULT_DTYPE)
        for s in range(0, n, self.max_batch):
            e = min(n, s + self.max_batch)
            ccst_track_host(self.ctx, frames_np[s:e], e - s, 0, res[s:e])
        return res


def decode(out) -> np.ndarray:
    """(n, 24) uint8 tensor/array of records -> numpy structured array."""
    a = out.cpu().numpy() if hasattr(out, "cpu") else np.asarray(out)
    return np.ascontiguousarray(a).view(RESULT_DTYPE).reshape(-1)
