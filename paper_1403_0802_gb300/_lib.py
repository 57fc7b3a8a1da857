"""ctypes loader of the in-tree libsj.so (the C ABI declared in include/sj.h).

The library must have been built (``paper_1403_0802_gb300.build.build()`` or
``__graft_entry__.build()``); there is no fallback: loading fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from .build import SO

_lock = threading.Lock()
_lib = None


class sj_grid(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("x1", C.c_double), ("y1", C.c_double),
                ("nx", C.c_int32), ("ny", C.c_int32)]


class sj_opts(C.Structure):
    _fields_ = [("form", C.c_int32), ("launch", C.c_int32), ("block", C.c_int32), ("pts_per_item", C.c_int32),
                ("edges_per_chunk", C.c_int32), ("flags", C.c_int32)]


class sj_layer_info(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_objects", C.c_int32), ("n_vertices", C.c_int64), ("n_rings", C.c_int64),
                ("n_cells", C.c_int64), ("n_candidates", C.c_int64), ("D", C.c_double)]


class sj_run_stats(C.Structure):
    _fields_ = [("joins", C.c_int64), ("points", C.c_int64), ("items", C.c_int64), ("pairs", C.c_int64),
                ("edge_tests", C.c_int64), ("fallbacks", C.c_int64), ("hits", C.c_int64),
                ("refine_launches", C.c_int64), ("refine_ms", C.c_double), ("algo_tests", C.c_int64),
                ("census_tests", C.c_int64), ("census_straddles", C.c_int64), ("resolved", C.c_int64)]


class sj_peak_rates(C.Structure):
    _fields_ = [("sms", C.c_int32), ("pad", C.c_int32), ("ffma_per_s", C.c_double), ("ffma_per_clk_sm", C.c_double),
                ("fadd_per_s", C.c_double), ("fadd_per_clk_sm", C.c_double), ("dfma_per_s", C.c_double),
                ("dfma_per_clk_sm", C.c_double), ("dadd_per_s", C.c_double), ("dadd_per_clk_sm", C.c_double)]


class sj_request(C.Structure):
    _fields_ = [("layer", C.c_void_p), ("pts", C.c_void_p), ("N", C.c_int64), ("out_id", C.c_void_p),
                ("out_d", C.c_void_p), ("use_window", C.c_int32), ("pad", C.c_int32), ("window", C.c_double)]


class sj_serve_request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("use_window", C.c_int32), ("pts", C.c_void_p), ("n", C.c_int64),
                ("out_id", C.c_void_p), ("out_d", C.c_void_p), ("not_before", C.c_double), ("window", C.c_double)]


class sj_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("rounds", C.c_int64), ("points", C.c_int64),
                ("max_launch_s", C.c_double), ("max_round_s", C.c_double)]


SJ_OK, SJ_ERR_INVALID, SJ_ERR_OOM, SJ_ERR_GRID_COVER, SJ_ERR_CUDA, SJ_ERR_TIMEOUT, SJ_ERR_BUSY = 0, -1, -2, -3, -4, -5, -6
SJ_ERR_CANCELLED = -7
SJ_FAULT_NONE, SJ_FAULT_ALLOC, SJ_FAULT_ADMIT = 0, 1, 2
SJ_FP64, SJ_FP32X = 0, 1
SJ_PER_REQUEST, SJ_PERSISTENT = 0, 1
SJ_FLAG_TIME_REFINE = 1
SJ_FLAG_NO_GRAPH = 2
SJ_FLAG_SUBCELL_ON = 4
SJ_FLAG_SUBCELL_OFF = 8
SJ_SERVE_BATCHED, SJ_SERVE_PER_REQUEST = 0, 1
SJ_SERVE_PIP, SJ_SERVE_P2P = 0, 1

# name -> (restype, argtypes); every name here is declared in include/*.h
_P, _I32, _I64, _D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
_LP = C.POINTER(C.c_void_p)
SIGNATURES = {
    "sj_pip_layer_create": (C.c_int, [_P, _I64, _P, _I64, _P, _I32, C.POINTER(sj_grid), _P, _LP]),
    "sj_p2p_layer_create": (C.c_int, [_P, _I64, _P, _I32, _D, C.POINTER(sj_grid), _P, _LP]),
    "sj_layer_destroy": (C.c_int, [_P]),
    "sj_layer_get_info": (C.c_int, [_P, C.POINTER(sj_layer_info)]),
    "sj_layer_get_candidates": (C.c_int, [_P, _P, _P]),
    "sj_pip_join": (C.c_int, [_P, _P, _I64, _P, C.POINTER(sj_opts), _P]),
    "sj_p2p_join": (C.c_int, [_P, _P, _I64, _P, _P, C.POINTER(sj_opts), _P]),
    "sj_p2p_join_window": (C.c_int, [_P, _P, _I64, C.c_double, _P, _P, C.POINTER(sj_opts), _P]),
    "sj_pip_join_host": (C.c_int, [_P, _P, _I64, _P, C.POINTER(sj_opts), _P]),
    "sj_p2p_join_host": (C.c_int, [_P, _P, _I64, _P, _P, C.POINTER(sj_opts), _P]),
    "sj_p2p_join_window_host": (C.c_int, [_P, _P, _I64, C.c_double, _P, _P, C.POINTER(sj_opts), _P]),
    "sj_p2p_join_noalloc": (C.c_int, [_P, _P, _I64, _P, _P, C.POINTER(sj_opts), _P]),
    "sj_bucket_points": (C.c_int, [_P, _I64, C.POINTER(sj_grid), _P, _P, _P]),
    "sj_layer_get_stats": (C.c_int, [_P, C.POINTER(sj_run_stats)]),
    "sj_pip_census": (C.c_int, [_P, _P, _I64, _P, _P]),
    "sj_layer_reset_stats": (C.c_int, [_P]),
    "sj_last_error": (C.c_char_p, []),
    "sj_version": (C.c_char_p, []),
    "sj_peaks_measure": (C.c_int, [C.POINTER(sj_peak_rates)]),
    "sj_engine_create": (C.c_int, [_I64, _I32, C.POINTER(sj_opts), _LP]),
    "sj_engine_round": (C.c_int, [_P, C.POINTER(sj_request), _I32, _P]),
    "sj_engine_destroy": (C.c_int, [_P]),
    "sj_server_create": (C.c_int, [_P, _P, C.POINTER(sj_opts), _I32, _I64, _I64, _I32, _LP]),
    "sj_server_submit": (C.c_int, [_P, C.POINTER(sj_serve_request), C.POINTER(C.c_int64)]),
    "sj_server_wait": (C.c_int, [_P, _I64, C.POINTER(C.c_double)]),
    "sj_server_wait_for": (C.c_int, [_P, _I64, _D, C.POINTER(C.c_double)]),
    "sj_server_cancel": (C.c_int, [_P, _I64]),
    "sj_fault_inject": (C.c_int, [_I32, _I32, _I32]),
    "sj_fault_pending": (C.c_int32, []),
    "sj_bounds_checked": (C.c_int32, []),
    "sj_server_poll": (C.c_int, [_P, _I64, C.POINTER(C.c_int32)]),
    "sj_server_drain": (C.c_int, [_P]),
    "sj_server_set_mode": (C.c_int, [_P, _I32, _I32]),
    "sj_server_get_stats": (C.c_int, [_P, C.POINTER(sj_server_stats)]),
    "sj_server_now": (C.c_double, [_P]),
    "sj_server_reset_maxima": (C.c_int, [_P]),
    "sj_server_destroy": (C.c_int, [_P]),
}


class SJError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


def use(path: str):
    """Load the library from `path` (for example the bounds-checked build)
    instead of the default one; only before the first call."""
    global SO
    with _lock:
        if _lib is not None and path != SO:
            raise RuntimeError("libsj.so is already loaded from " + SO)
        SO = path


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(SO):
                raise RuntimeError(f"libsj.so is not built ({SO}); run paper_1403_0802_gb300.build.build()")
            L = C.CDLL(SO)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def check(status: int, where: str):
    if status != SJ_OK:
        raise SJError(status, where, lib().sj_last_error().decode())
