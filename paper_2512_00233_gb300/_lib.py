"""ctypes declarations of the C ABI in include/kcore.h.

Loads libkcore.so from this package directory (building it with nvcc when it
is missing or stale).  There is no fallback: if the library cannot be built
or loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

c_i32, c_i64, c_u32, c_u64, c_vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                    ctypes.c_uint64, ctypes.c_void_p)

KCORE_OK = 0
KCORE_PENDING = 1
KCORE_ERR_INVALID = -1
KCORE_ERR_OOM = -2
KCORE_ERR_CUDA = -3
KCORE_ERR_NOT_CONVERGED = -4
KCORE_ERR_TIMEOUT = -5
KCORE_ERR_AGAIN = -6
KCORE_ERR_CANCELLED = -7

KCORE_IN_DEVICE = 1 << 0
KCORE_IN_CLEAN = 1 << 1
KCORE_OUT_DEVICE = 1 << 2
KCORE_SYNC_MODE = 1 << 3
KCORE_REFINED = 1 << 4
KCORE_ASYNC = 1 << 5
KCORE_GRAPH = 1 << 6
KCORE_SIMPLE = 1 << 7

KCORE_NOALLOC_MAX_N = 1 << 19

STATUS_NAMES = {
    KCORE_OK: "OK", KCORE_PENDING: "PENDING", KCORE_ERR_INVALID: "ERR_INVALID",
    KCORE_ERR_OOM: "ERR_OOM", KCORE_ERR_CUDA: "ERR_CUDA",
    KCORE_ERR_NOT_CONVERGED: "ERR_NOT_CONVERGED", KCORE_ERR_TIMEOUT: "ERR_TIMEOUT",
    KCORE_ERR_AGAIN: "ERR_AGAIN", KCORE_ERR_CANCELLED: "ERR_CANCELLED",
}


class Options(ctypes.Structure):
    _fields_ = [("struct_size", c_u32), ("t_lo", c_i32), ("t_hi", c_i32), ("block", c_i32),
                ("low_chunk", c_i32), ("med_chunk", c_i32), ("tail_max", c_i32),
                ("ctas_per_sm", c_i32), ("max_ctas", c_i32), ("max_sweeps", c_i64),
                ("timeout_s", ctypes.c_double), ("build_sort", c_i32), ("relabel", c_i32)]


class RunStats(ctypes.Structure):
    _fields_ = [("n", c_i64), ("nnz", c_i64), ("sweeps", c_i64), ("tail_sweeps", c_i64),
                ("evaluated", c_i64), ("edges_scanned", c_i64), ("updates", c_i64),
                ("pushes", c_i64), ("bytes_algorithmic", c_i64), ("status", c_i32),
                ("grid", c_i32), ("block", c_i32), ("row_ptr_bytes", c_i32),
                ("ms_create", ctypes.c_float), ("ms_sweep", ctypes.c_float),
                ("ms_run", ctypes.c_float), ("entries_read", c_i64), ("decrease", c_i64)]


class ServeOptions(ctypes.Structure):
    _fields_ = [("struct_size", c_u32), ("mem_budget", c_i64), ("max_slots", c_i32),
                ("max_queue", c_i32), ("chunk_sweeps", c_i32), ("start_thread", c_i32),
                ("sweep", Options), ("host_staging", c_i64)]


class BatchStats(ctypes.Structure):
    _fields_ = [("submitted", c_i64), ("completed", c_i64), ("cancelled", c_i64),
                ("failed", c_i64), ("queued", c_i64), ("resident", c_i64),
                ("launches", c_i64), ("sweeps", c_i64), ("arena_bytes", c_i64),
                ("arena_used_peak", c_i64), ("latency_p50_ms", ctypes.c_double),
                ("latency_p99_ms", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("sweep_s", ctypes.c_double),
                ("retire_s", ctypes.c_double), ("admissions", c_i64),
                ("admitted_while_busy", c_i64)]


class TicketInfo(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("admit_launch", c_i64), ("retire_launch", c_i64),
                ("resident_at_admit", c_i64)]


# name: (restype, argtypes)
SIGNATURES = {
    "kcore_default_options": (None, [ctypes.POINTER(Options)]),
    "kcore_create": (c_i32, [c_i64, c_vp, c_i32, c_vp, c_u32, ctypes.POINTER(Options), c_vp,
                             ctypes.POINTER(c_vp)]),
    "kcore_create_coo": (c_i32, [c_i64, c_i64, c_vp, c_vp, c_i32, c_u32, ctypes.POINTER(Options),
                                 c_vp, ctypes.POINTER(c_vp)]),
    "kcore_set_options": (c_i32, [c_vp, ctypes.POINTER(Options), c_vp]),
    "kcore_run": (c_i32, [c_vp, c_vp, c_u32, c_vp]),
    "kcore_wait": (c_i32, [c_vp]),
    "kcore_graph_info": (c_i32, [c_vp, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64),
                                 ctypes.POINTER(c_i32)]),
    "kcore_copy_csr": (c_i32, [c_vp, c_vp, c_vp, c_u32]),
    "kcore_stats": (c_i32, [c_vp, ctypes.POINTER(RunStats)]),
    "kcore_sweep_trace": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(c_i64)]),
    "kcore_sweep_detail": (c_i32, [c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(c_i64)]),
    "kcore_sweep_tiers": (c_i32, [c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(c_i64)]),
    "kcore_run_from": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_vp, c_u32, c_vp]),
    "kcore_destroy": (None, [c_vp]),
    "kcore_run_noalloc": (c_i32, [c_i64, c_vp, c_i32, c_vp, c_vp, c_vp]),
    "kcore_default_serve_options": (None, [ctypes.POINTER(ServeOptions)]),
    "kcore_batch_create": (c_i32, [ctypes.POINTER(ServeOptions), ctypes.POINTER(c_vp)]),
    "kcore_submit": (c_i32, [c_vp, c_i64, c_vp, c_i32, c_vp, c_u32, ctypes.POINTER(c_u64)]),
    "kcore_submit_coo": (c_i32, [c_vp, c_i64, c_i64, c_vp, c_vp, c_u32, ctypes.POINTER(c_u64)]),
    "kcore_poll": (c_i32, [c_vp, c_u64, c_vp, c_i64]),
    "kcore_poll_info": (c_i32, [c_vp, c_u64, c_vp, c_i64, ctypes.POINTER(TicketInfo)]),
    "kcore_cancel": (c_i32, [c_vp, c_u64]),
    "kcore_batch_step": (c_i32, [c_vp, ctypes.POINTER(c_i64)]),
    "kcore_batch_stats_get": (c_i32, [c_vp, ctypes.POINTER(BatchStats)]),
    "kcore_batch_destroy": (None, [c_vp]),
    "kcore_last_error": (ctypes.c_char_p, []),
    "kcore_version": (ctypes.c_char_p, []),
    "kcore_kernel_launches": (c_i64, []),
    "kcore_release_cached_memory": (None, []),
    # test hooks (include/kcore_test.h)
    "kcore_test_fail_alloc": (None, [c_i64]),
    "kcore_test_alloc_count": (c_i64, []),
    "kcore_test_pool_usage": (c_i32, [ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
}

_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """The loaded libkcore.so (built on first use if needed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libkcore.so is missing and could not be built")
            handle = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
        return _lib


class KCoreError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().kcore_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str) -> int:
    if status < 0:
        raise KCoreError(status, where)
    return status
