"""ctypes declarations of the C ABI in ``include/propagate.h``.

Argument marshalling only: every step of the propagation runs in the CUDA
library. Loading fails loudly if the library cannot be built or found.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PG_OK, PG_EINVAL, PG_ENOMEM, PG_ECUDA, PG_ETIMEOUT, PG_EDEVICE, PG_ECANCELLED, PG_ERANGE = (
    0, -1, -2, -3, -4, -5, -6, -7)
PG_ETOOBIG = -8
PG_NOALLOC_SCRATCH_BYTES = 32 << 20
PG_NOALLOC_MAX_SEEDS = 1024
PG_DEVICE_PTRS = 1
PG_BORROW = 2
PG_REVERSE = 4
PG_RELABEL = 8
PG_KEEP_ORDER = 16
PG_HOST_CSR = 32
PG_DIR_AUTO, PG_DIR_DENSE, PG_DIR_SPARSE = 0, 1, 2
PG_ALG_P, PG_ALG_S = 0, 1


class Options(ctypes.Structure):
    _fields_ = [("direction", ctypes.c_int32), ("dense_threshold", ctypes.c_float),
                ("group_lanes", ctypes.c_int32),
                ("test_changed", ctypes.c_int32), ("planes_per_pass", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("window_rows", ctypes.c_int32), ("words_per_thread", ctypes.c_int32),
                ("wide_rows", ctypes.c_int32), ("passes_together", ctypes.c_int32),
                ("pass_words", ctypes.c_int32), ("tma_gather", ctypes.c_int32),
                ("sparse_push", ctypes.c_int32)]


class Generator(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("directed", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("n", ctypes.c_int64),
                ("avg_degree", ctypes.c_double), ("scale", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("edge_factor", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double),
                ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("p_delete", ctypes.c_double)]


PG_GEN_ER, PG_GEN_RMAT, PG_GEN_GRID = 0, 1, 2


class Counts(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int32), ("max_rounds", ctypes.c_int32),
                ("rounds", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("counts", ctypes.c_void_p), ("m_active", ctypes.c_void_p)]


class MetricsOut(ctypes.Structure):
    _fields_ = [("diameter", ctypes.c_int32), ("eff_diameter", ctypes.c_int32),
                ("eff_diameter_interp", ctypes.c_double), ("avg_distance", ctypes.c_double),
                ("avg_distance_incl_self", ctypes.c_double),
                ("connectivity_rate", ctypes.c_double), ("reachable_pairs", ctypes.c_double),
                ("R_last", ctypes.c_uint64), ("dist_sum", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("dense_rounds", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("m_active_total", ctypes.c_uint64), ("arcs_scanned", ctypes.c_uint64),
                ("rows_gathered", ctypes.c_uint64), ("items", ctypes.c_uint64),
                ("changed_rows", ctypes.c_uint64), ("frontier_arcs", ctypes.c_uint64),
                ("words_per_row", ctypes.c_int32), ("group_lanes", ctypes.c_int32),
                ("ms_pull", ctypes.c_double), ("ms_post", ctypes.c_double),
                ("ms_init", ctypes.c_double), ("pull_launches", ctypes.c_int32),
                ("post_launches", ctypes.c_int32), ("test_changed", ctypes.c_int32),
                ("words_per_gather", ctypes.c_int32), ("seed_edge_traversals", ctypes.c_uint64),
                ("pass_words", ctypes.c_int32), ("dense_tma", ctypes.c_int32),
                ("active_rows", ctypes.c_uint64)]


class TuneReport(ctypes.Structure):
    _fields_ = [("trials", ctypes.c_int32), ("improved", ctypes.c_int32),
                ("default_ms", ctypes.c_double), ("best_ms", ctypes.c_double)]


class BatchStats(ctypes.Structure):
    _fields_ = [("graphs", ctypes.c_int32), ("groups", ctypes.c_int32),
                ("sweeps", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("seed_edge_traversals", ctypes.c_uint64)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("merge_max", ctypes.c_int32),
                ("merge_max_seeds", ctypes.c_int32), ("cross_graph", ctypes.c_int32),
                ("hbm_budget", ctypes.c_int64), ("opt", Options)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32),
                ("rounds", ctypes.c_int32), ("s", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("merged", ctypes.c_int32), ("footprint", ctypes.c_int64),
                ("submit_ns", ctypes.c_int64), ("start_ns", ctypes.c_int64),
                ("done_ns", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("propagations", ctypes.c_int64), ("resident_bytes", ctypes.c_int64),
                ("inflight_bytes", ctypes.c_int64), ("peak_bytes", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64), ("graphs", ctypes.c_int32),
                ("queued", ctypes.c_int32), ("running", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("seed_edge_traversals", ctypes.c_uint64),
                ("gpu_launches", ctypes.c_int64)]


PG_REQ_QUEUED, PG_REQ_RUNNING, PG_REQ_DONE, PG_REQ_FAILED, PG_REQ_CANCELLED = 0, 1, 2, 3, 4


# name -> (restype, argtypes); every symbol declared in include/propagate.h
_vp, _i32, _i64, _u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
SIGNATURES = {
    "pg_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "pg_version": (ctypes.c_char_p, []),
    "pg_default_options": (None, [ctypes.POINTER(Options)]),
    "pg_graph_from_csr": (ctypes.c_int, [_vp, _vp, _i64, _i64, ctypes.c_int, ctypes.c_uint,
                                         _vp, ctypes.POINTER(_vp)]),
    "pg_graph_free": (None, [_vp]),
    "pg_graph_info": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "pg_graph_is_relabelled": (ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    "pg_graph_generate": (ctypes.c_int, [ctypes.POINTER(Generator), ctypes.c_uint, _vp,
                                         ctypes.POINTER(_vp)]),
    "pg_graph_copy_csr": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "pg_query_rounds_bound": (ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    "pg_propagate_p": (ctypes.c_int, [_vp, _vp, _i32, ctypes.POINTER(Counts),
                                      ctypes.POINTER(Options), _vp]),
    "pg_propagate_s": (ctypes.c_int, [_vp, _vp, _i32, ctypes.POINTER(Counts),
                                      ctypes.POINTER(Options), _vp]),
    "pg_metrics": (ctypes.c_int, [ctypes.POINTER(Counts), _i64, _i32, _i32,
                                  ctypes.POINTER(MetricsOut)]),
    "pg_last_stats": (ctypes.c_int, [_vp, ctypes.POINTER(Stats)]),
    "pg_progressive": (ctypes.c_int, [_vp, ctypes.c_double, _i32, ctypes.c_double,
                                      ctypes.c_uint64, _vp, ctypes.POINTER(_i32),
                                      ctypes.POINTER(Counts), ctypes.POINTER(MetricsOut), _i32,
                                      ctypes.POINTER(_i32), ctypes.POINTER(Options), _vp]),
    "pg_propagate_p_noalloc": (ctypes.c_int, [_vp, _vp, _i64, _i64, _vp, _i32, _vp, _i32,
                                              ctypes.POINTER(_i32), _vp]),
    "pg_autotune": (ctypes.c_int, [_vp, _vp, _i32, _i32, _i32, ctypes.POINTER(Options),
                                   ctypes.POINTER(TuneReport), _vp]),
    "pg_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp)]),
    "pg_batch_free": (None, [_vp]),
    "pg_batch_add": (ctypes.c_int, [_vp, _vp, _vp, _i64, _i64, ctypes.c_int, _vp, _i32,
                                    ctypes.POINTER(_i32)]),
    "pg_batch_run": (ctypes.c_int, [_vp, ctypes.POINTER(Options), _vp]),
    "pg_batch_result": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(Counts)]),
    "pg_batch_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(BatchStats)]),
    "pg_batch_tune": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(TuneReport), _vp]),
    "pg_batch_group_stats": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(Stats)]),
    "pg_batch_set_streams": (ctypes.c_int, [_vp, _i32]),
    "pg_batch_get_options": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(Options),
                                            ctypes.POINTER(_i32)]),
    "pg_server_default_config": (None, [ctypes.POINTER(ServerConfig)]),
    "pg_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_vp)]),
    "pg_server_destroy": (None, [_vp]),
    "pg_server_add_graph": (ctypes.c_int, [_vp, _vp, _vp, _i64, _i64, ctypes.c_int,
                                           ctypes.POINTER(_i32)]),
    "pg_server_remove_graph": (ctypes.c_int, [_vp, _i32]),
    "pg_server_submit": (ctypes.c_int, [_vp, _i32, _vp, _i32, ctypes.POINTER(_i64)]),
    "pg_server_poll": (ctypes.c_int, [_vp, _i64, ctypes.POINTER(RequestInfo)]),
    "pg_server_wait": (ctypes.c_int, [_vp, _i64, _i32, ctypes.POINTER(RequestInfo)]),
    "pg_server_result": (ctypes.c_int, [_vp, _i64, ctypes.POINTER(Counts),
                                        ctypes.POINTER(RequestInfo)]),
    "pg_server_cancel": (ctypes.c_int, [_vp, _i64]),
    "pg_server_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ServerStats)]),
}

_lock = threading.Lock()
_lib = None


def lib():
    """The loaded CUDA library (built in-tree on first use if missing). The
    environment variable PG_LIBRARY_VARIANT=debug-bounds selects the build
    whose gathers check their indices."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(variant=os.environ.get("PG_LIBRARY_VARIANT", ""))
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class PropagateError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = lib().pg_strerror(status).decode()
        super().__init__(f"{what}: {msg} (status {status})")
        self.status = status


def check(status: int, what: str):
    if status != PG_OK:
        raise PropagateError(status, what)
