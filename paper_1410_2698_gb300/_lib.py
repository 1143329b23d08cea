"""ctypes declarations of the C ABI in include/ts.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

_lock = threading.Lock()
_lib = None

TS_OK = 0
STATUS_NAMES = {0: "TS_OK", 1: "TS_ERR_INVALID_ARG", 2: "TS_ERR_OOM", 3: "TS_ERR_CUDA",
                4: "TS_ERR_CAPACITY", 5: "TS_ERR_TIMEOUT", 6: "TS_ERR_CANCELLED",
                7: "TS_ERR_INTERNAL"}

KINDS = {"brute": 0, "spatial": 1, "temporal": 2, "spatiotemporal": 3}

FIELDS = {"perm": 0, "bin_start": 1, "bin_end": 2, "bin_off": 3, "st_ids": 4, "st_off": 5,
          "grid_a": 6, "grid_off": 7}


class TsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ts_segments(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_void_p), ("y0", ctypes.c_void_p), ("z0", ctypes.c_void_p),
                ("t0", ctypes.c_void_p), ("x1", ctypes.c_void_p), ("y1", ctypes.c_void_p),
                ("z1", ctypes.c_void_p), ("t1", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("on_host", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ts_index_params(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("t_bins", ctypes.c_uint32),
                ("sub_bins", ctypes.c_uint32), ("grid_cells", ctypes.c_uint32)]


class ts_query_params(ctypes.Structure):
    _fields_ = [("d", ctypes.c_double), ("t_start", ctypes.c_double), ("t_end", ctypes.c_double),
                ("max_results", ctypes.c_uint64)]


class ts_search_stats(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_uint64), ("n_qsegs", ctypes.c_uint64),
                ("n_tests", ctypes.c_uint64), ("n_exact", ctypes.c_uint64),
                ("n_hits", ctypes.c_uint64), ("n_tiles", ctypes.c_uint64),
                ("n_groups", ctypes.c_uint64), ("n_subbin", ctypes.c_uint64),
                ("ms_count_pass", ctypes.c_double), ("ms_write_pass", ctypes.c_double),
                ("n_chunks", ctypes.c_uint64), ("n_dense", ctypes.c_uint64),
                ("n_sparse", ctypes.c_uint64), ("n_stage2", ctypes.c_uint64)]

    def as_dict(self):
        return {k: (float(getattr(self, k)) if k.startswith("ms_") else int(getattr(self, k)))
                for k, _ in self._fields_}


class ts_index_info(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("t_bins", ctypes.c_uint32),
                ("sub_bins", ctypes.c_uint32 * 3), ("grid_cells", ctypes.c_uint32),
                ("n", ctypes.c_uint64), ("st_len", ctypes.c_uint64 * 3),
                ("grid_len", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("t_min", ctypes.c_double), ("t_max", ctypes.c_double),
                ("bin_width", ctypes.c_double), ("sub_lo", ctypes.c_double * 3),
                ("sub_w", ctypes.c_double * 3), ("grid_lo", ctypes.c_double * 3),
                ("grid_w", ctypes.c_double * 3)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if hasattr(v, "__len__") else v
        return out


class ts_batch_params(ctypes.Structure):
    _fields_ = [("max_requests", ctypes.c_uint32), ("tile_records", ctypes.c_uint32),
                ("max_queries", ctypes.c_uint64), ("max_rows", ctypes.c_uint64),
                ("max_units", ctypes.c_uint64), ("max_tiles", ctypes.c_uint64),
                ("use_graph", ctypes.c_int32), ("pair_blocks", ctypes.c_int32),
                ("scratch_rows", ctypes.c_uint64)]


class ts_batch_status(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_uint64), ("nreq", ctypes.c_uint32),
                ("overflow", ctypes.c_int32), ("stats", ts_search_stats)]


class ts_server_params(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_uint32), ("max_batch_requests", ctypes.c_uint32),
                ("max_batch_queries", ctypes.c_uint64), ("max_batch_rows", ctypes.c_uint64),
                ("tile_records", ctypes.c_uint32), ("use_graph", ctypes.c_int32),
                ("linger_us", ctypes.c_uint32), ("admit_wait_ms", ctypes.c_uint32),
                ("scratch_rows", ctypes.c_uint64), ("mem_budget_bytes", ctypes.c_uint64)]


class ts_request_timing(ctypes.Structure):
    _fields_ = [("submit_us", ctypes.c_double), ("start_us", ctypes.c_double),
                ("done_us", ctypes.c_double), ("batch_requests", ctypes.c_uint32),
                ("requeued", ctypes.c_uint32)]


_P = ctypes.c_void_p
_S = ctypes.c_int
# name -> (restype, argtypes); every symbol declared in include/ts.h
SIGNATURES = {
    "ts_build_index": (_S, [ctypes.POINTER(ts_segments), ctypes.POINTER(ts_index_params), _P,
                            ctypes.POINTER(_P)]),
    "ts_index_get_info": (_S, [_P, ctypes.POINTER(ts_index_info)]),
    "ts_index_export": (_S, [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_uint64,
                             ctypes.POINTER(ctypes.c_uint64)]),
    "ts_schedule": (_S, [_P, ctypes.POINTER(ts_segments), ctypes.POINTER(ts_query_params), _P,
                         _P, _P, _P]),
    "ts_search": (_S, [_P, ctypes.POINTER(ts_segments), ctypes.POINTER(ts_query_params), _P,
                       ctypes.POINTER(_P)]),
    "ts_measure_alu_peaks": (_S, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "ts_eval_refined_estimates": (_S, [_P, ctypes.c_uint64, _P, _P, _P, _P]),
    "ts_debug_inject_stall": (_S, [ctypes.c_uint64]),
    "ts_search_points": (_S, [_P, _P, _P, _P, ctypes.c_uint64, ctypes.c_int32,
                              ctypes.POINTER(ts_query_params), _P, ctypes.POINTER(_P)]),
    "ts_result_count": (ctypes.c_uint64, [_P]),
    "ts_result_arrays": (_S, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                              ctypes.POINTER(_P)]),
    "ts_result_stats": (_S, [_P, ctypes.POINTER(ts_search_stats)]),
    "ts_result_copy_to_host": (_S, [_P, _P, _P, _P, _P, _P]),
    "ts_free": (None, [_P]),
    "ts_last_error": (ctypes.c_char_p, []),
    "ts_version": (ctypes.c_char_p, []),
    "ts_kernel_launches": (ctypes.c_uint64, []),
    "ts_search_batch": (_S, [_P, ctypes.c_uint32, ctypes.POINTER(ts_segments),
                             ctypes.POINTER(ts_query_params), _P, ctypes.POINTER(_P)]),
    "ts_batch_create": (_S, [_P, ctypes.POINTER(ts_batch_params), _P, ctypes.POINTER(_P)]),
    "ts_batch_run": (_S, [_P, ctypes.c_uint32, ctypes.POINTER(ts_segments),
                          ctypes.POINTER(ts_query_params), _P]),
    "ts_batch_wait": (_S, [_P, ctypes.POINTER(ts_batch_status)]),
    "ts_batch_request_rows": (_S, [_P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                   ctypes.POINTER(ctypes.c_uint64)]),
    "ts_batch_rows": (_S, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                           ctypes.POINTER(_P)]),
    "ts_batch_copy_rows": (_S, [_P, ctypes.c_uint64, ctypes.c_uint64, _P, _P, _P, _P]),
    "ts_server_create": (_S, [_P, ctypes.POINTER(ts_server_params), ctypes.POINTER(_P)]),
    "ts_server_info": (_S, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                            ctypes.POINTER(ctypes.c_uint64)]),
    "ts_server_submit": (_S, [_P, ctypes.POINTER(ts_segments), ctypes.POINTER(ts_query_params),
                              ctypes.POINTER(ctypes.c_uint64)]),
    "ts_server_wait": (_S, [_P, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(_P),
                            ctypes.POINTER(ts_request_timing)]),
    "ts_server_cancel": (_S, [_P, ctypes.c_uint64]),
    "ts_server_destroy": (None, [_P]),
    "ts_search_brute_noalloc": (_S, [ctypes.POINTER(ts_segments), ctypes.POINTER(ts_segments),
                                     ctypes.POINTER(ts_query_params), _P, _P, _P, _P,
                                     ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), _P]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libts_gb300.so (building it first when missing). Raises if it cannot be loaded:
    there is no fallback implementation."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path}")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int):
    if status != TS_OK:
        msg = _lib.ts_last_error().decode() if _lib is not None else ""
        raise TsError(status, msg)
