"""B300-native cross-correlation sub-pixel tracking (arXiv 2310.08770).

The compute path lives in the CUDA library ``libccst.so`` (built from
``csrc/``); :mod:`.ccst` is a thin ctypes binding to its C ABI. Importing the
package does not load the library: the first call that needs it does, and it
raises if the library is missing.
"""
_BINDING = ("CC_SN", "CC_U", "Tracker", "CcstError", "RESULT_DTYPE", "decode", "library_path",
            "ccst_version", "ccst_default_params", "ccst_create", "ccst_track", "ccst_track_host",
            "ccst_set_stream", "ccst_sync", "ccst_submit", "ccst_poll", "ccst_backward",
            "ccst_destroy", "ccst_grid_size", "ccst_debug_surfaces", "ccst_profile_kernel_ms",
            "ccst_profile_reset", "ccst_debug_pairs", "ccst_track_static",
            "ccst_rt_begin", "ccst_rt_track", "ccst_drift_correct", "ccst_set_reference_frame",
            "ccst_offline_update", "ccst_offline_track", "ccst_reference_status", "ccst_peak_continuous",
            "ccst_add_reference", "ccst_track_rois", "make_rois", "ccst_server_create", "ccst_server_submit",
            "ccst_server_poll", "ccst_server_read_stats", "ccst_server_loadgen", "ccst_server_destroy")


def __getattr__(name):
    if name in _BINDING:
        from . import ccst
        return getattr(ccst, name)
    raise AttributeError(name)
