"""ctypes binding of ``libsvt.so`` (the C ABI in include/svt.h).

Argument marshalling only: every function here forwards to the CUDA library
and raises when it reports a host-side error.  There is no CPU fallback: if
the library is missing the import of the binding fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsvt.so")

SVT_OK = 0
ERRORS = {
    1: "BAD_ARG", 2: "BAD_TYPE", 3: "BAD_RESERVED", 4: "BAD_LAYER", 5: "UNSORTED",
    6: "TOO_MANY_HITS", 7: "BAD_SECTOR", 8: "NROADS_MISMATCH", 9: "OOM", 10: "BAD_CONFIG",
    11: "TIMEOUT", 12: "XFT_UNPAIRED", 20: "CUDA",
}
STATUS_OK = (1 << 64) - 1
FLAG_PASS, FLAG_OVERFLOW, FLAG_BAD_PATTERN, FLAG_NO_HITS = 1, 2, 4, 8


class SvtError(RuntimeError):
    pass


class SvtConfig(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("oshift", "qshift", "chi2_cut", "max_comb", "min_layers", "n_sectors",
                 "xft_pairs")]


class SvtSchedule(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("warps_per_block", "blocks_per_sm", "rows_per_item", "roads_per_chunk",
                 "small_max", "pair_small")]


class SvtServerConfig(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_uint32), ("mode", ctypes.c_uint32),
                ("max_words", ctypes.c_uint64), ("max_events", ctypes.c_uint64),
                ("max_roads", ctypes.c_uint64), ("max_combs", ctypes.c_uint64),
                ("device_budget", ctypes.c_uint64), ("max_queued_words", ctypes.c_uint64),
                ("small_batch_events", ctypes.c_uint32), ("small_blocks_per_sm", ctypes.c_uint32)]


class SvtEventResult(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_uint64), ("n_roads", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("latency_ns", ctypes.c_uint64),
                ("t_arrive_ns", ctypes.c_int64)]


class SvtServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("batches", "events_done", "events_failed", "retried_batches", "rejected", "queued",
                 "h2d_bytes", "d2h_bytes", "max_queued", "max_batch_events", "launch_ns",
                 "finish_ns")]


class SvtBatchTrace(ctypes.Structure):
    _fields_ = [("slot", ctypes.c_uint32), ("n_events", ctypes.c_uint32),
                ("n_roads", ctypes.c_uint32), ("queued_after", ctypes.c_uint32),
                ("t_first_arrive_ns", ctypes.c_int64), ("t_dispatch_ns", ctypes.c_int64),
                ("t_enqueued_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64),
                ("dev_start_us", ctypes.c_float), ("dev_end_us", ctypes.c_float)]


class SvtBest(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("comb", ctypes.c_uint32), ("chi2", ctypes.c_uint32),
                ("p", ctypes.c_int32 * 3)]


_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_sz = ctypes.c_size_t
_cfgp = ctypes.POINTER(SvtConfig)
_schp = ctypes.POINTER(SvtSchedule)

# name -> (restype, argtypes); mirrors include/svt.h
SIGNATURES = {
    "svt_version": (ctypes.c_int, []),
    "svt_device_sm_count": (ctypes.c_int, [ctypes.c_int]),
    "svt_pipe_peak": (ctypes.c_int, [_u32, _u32, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), _vp]),
    "svt_unpack_workspace_size": (_sz, [_u64]),
    "svt_unpack": (ctypes.c_int, [_vp, _u64, _vp, _u64, _u32, _u32, _u64, _vp, _vp, _vp, _vp,
                                  _vp, _vp, _sz, _vp]),
    "svt_combine_workspace_size": (_sz, [_u64]),
    "svt_combine": (ctypes.c_int, [_vp, _vp, _u64, _cfgp, _u64, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                   _sz, _vp]),
    "svt_fit": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _u64, _vp, _vp, _cfgp, _vp, _vp, _vp,
                               _vp]),
    "svt_select": (ctypes.c_int, [_vp, _vp, _u64, _vp, _vp, _vp, _u64, _cfgp, _vp, _vp, _vp]),
    "svt_format": (ctypes.c_int, [_vp, _vp, _vp, _vp, _u64, _vp, _vp, _vp]),
    "svt_run_workspace_size": (_sz, [_u64, _u64, _u64, _schp]),
    "svt_run": (ctypes.c_int, [_vp, _u64, _vp, _u64, _vp, _vp, _cfgp, _u64, _vp, _vp, _vp, _vp,
                               _vp, _sz, _schp, _vp, _vp]),
    "svt_run_sized": (ctypes.c_int, [_vp, _u64, _vp, _u64, _vp, _vp, _vp, _cfgp, _u64, _vp, _vp,
                                     _vp, _vp, _vp, _sz, _schp, _vp]),
    "svt_graph_create": (ctypes.c_int, [_vp, _u64, _vp, _u64, _vp, _vp, _vp, _cfgp, _u64, _vp,
                                        _vp, _vp, _vp, _vp, _sz, _schp, ctypes.POINTER(_vp)]),
    "svt_autotune": (ctypes.c_int, [_vp, _u64, _vp, _u64, _vp, _vp, _cfgp, _u64, _vp, _vp, _vp,
                                    _sz, _u32, _vp, _sz, _schp, ctypes.POINTER(ctypes.c_float),
                                    _vp]),
    "svt_graph_launch": (ctypes.c_int, [_vp, _vp]),
    "svt_graph_destroy": (ctypes.c_int, [_vp]),
    "svt_host_alloc": (ctypes.c_int, [_sz, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "svt_host_free": (ctypes.c_int, [_vp]),
    "svt_run_host_workspace_size": (_sz, [_u64, _u64, _u64, _schp]),
    "svt_run_host": (ctypes.c_int, [_vp, _u64, _vp, _u64, _vp, _vp, _cfgp, _u64, _vp, _vp,
                                    ctypes.POINTER(_u64), _vp, _sz, _schp, _vp]),
    "svt_run_noalloc_scratch_bytes": (_sz, []),
    "svt_run_noalloc": (ctypes.c_int, [_vp, _u64, _vp, _u64, _vp, _vp, _cfgp, _u64, _vp, _vp, _vp,
                                       _vp, _schp, _vp]),
    "svt_timer_create": (ctypes.c_int, [ctypes.POINTER(_vp)]),
    "svt_timer_destroy": (ctypes.c_int, [_vp]),
    "svt_timer_fit_ms": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float)]),
    "svt_server_sizes": (ctypes.c_int, [ctypes.POINTER(SvtServerConfig), _schp,
                                        ctypes.POINTER(_sz), ctypes.POINTER(_sz)]),
    "svt_server_create": (ctypes.c_int, [ctypes.POINTER(SvtServerConfig), _vp, _vp, _cfgp, _schp,
                                         _vp, _sz, _vp, _sz, ctypes.POINTER(_vp)]),
    "svt_server_submit": (ctypes.c_int, [_vp, _vp, _u32, _u64, _vp]),
    "svt_server_poll": (ctypes.c_int, [_vp, ctypes.POINTER(SvtEventResult), _u32,
                                       ctypes.POINTER(_u32), _u32]),
    "svt_server_stats_get": (ctypes.c_int, [_vp, ctypes.POINTER(SvtServerStats)]),
    "svt_server_stats_reset": (ctypes.c_int, [_vp]),
    "svt_server_trace": (ctypes.c_int, [_vp, _vp, _u64, _u32]),
    "svt_server_trace_count": (ctypes.c_int, [_vp, ctypes.POINTER(_u64)]),
    "svt_server_destroy": (ctypes.c_int, [_vp]),
    "svt_server_bench_poisson": (ctypes.c_int, [_vp, _vp, _vp, _u32, ctypes.c_double, _u64, _u64,
                                                _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double)]),
    "svt_calib_index_size": (_sz, [_u64, _u32]),
    "svt_calib_index": (ctypes.c_int, [_vp, _u64, _u32, _vp, _sz, _vp, _vp, _vp]),
    "svt_calib_gather": (ctypes.c_int, [_vp, _u32, _vp, _u64, _vp, _vp]),
    "svt_calib_workspace_size": (_sz, [_u64, _u32]),
    "svt_calib_forward": (ctypes.c_int, [_vp, _u64, _u32, _vp, _vp, _vp, _vp, _vp]),
    "svt_calib_loss": (ctypes.c_int, [_vp, _vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "svt_calib_loss_backward": (ctypes.c_int, [_vp, _vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp, _vp,
                                               _vp, _vp, _sz, _vp]),
    "svt_calib_backward": (ctypes.c_int, [_vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp, _vp, _vp, _sz,
                                          _vp]),
    "svt_calib_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp, _vp, _vp,
                                           _vp, _vp, _sz, _vp]),
    "svt_calib_grad_scale": (ctypes.c_int, [_vp, _vp, _vp, _u32, _vp, _vp, _vp]),
}

_lib = None
_lock = threading.Lock()


def load():
    """Load libsvt.so (building it first when nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            from . import build as _build
            try:
                _build.build()
            except Exception as e:  # noqa: BLE001
                raise ImportError(f"libsvt.so is missing and could not be built: {e}") from e
        else:
            from . import build as _build
            try:
                _build.build()   # rebuild when sources are newer
            except RuntimeError:
                pass
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return _lib


def check(rc: int, what: str):
    if rc != SVT_OK:
        raise SvtError(f"{what} failed: {ERRORS.get(rc, rc)}")


def decode_status(key: int):
    """(word_index, error name) of a device status key, or None when OK."""
    key = int(key) & STATUS_OK
    if key == STATUS_OK:
        return None
    return key >> 8, ERRORS.get(key & 0xFF, key & 0xFF)
