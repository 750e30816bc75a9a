"""GB300 k-core decomposition: Python binding of libkcore (include/kcore.h).

This layer only marshals arguments: numpy arrays are host pointers, CUDA
torch tensors are device pointers, and torch's current stream is passed as the
cudaStream_t.  Every step of the computation runs in the library's sm_103a
kernels; there is no Python or CPU fallback.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import (KCORE_ASYNC, KCORE_GRAPH, KCORE_SIMPLE, KCORE_ERR_AGAIN, KCORE_ERR_CANCELLED, KCORE_ERR_INVALID,
                   KCORE_ERR_OOM, KCORE_ERR_CUDA,
                   KCORE_ERR_NOT_CONVERGED, KCORE_ERR_TIMEOUT, KCORE_IN_CLEAN, KCORE_IN_DEVICE,
                   KCORE_OK, KCORE_OUT_DEVICE, KCORE_PENDING, KCORE_REFINED, KCORE_SYNC_MODE,
                   SIGNATURES, BatchStats, KCoreError, Options, RunStats, ServeOptions, TicketInfo,
                   check, lib)

__all__ = ["Graph", "BatchEngine", "default_options", "default_serve_options", "lib",
           "KCoreError", "Options", "RunStats", "TicketInfo", "version"]


def version() -> str:
    return lib().kcore_version().decode()


def _torch():
    import torch
    return torch


def _stream(stream) -> int:
    if stream is None:
        torch = _torch()
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


def _ptr(x, dtype):
    """(pointer, keepalive, is_device) of a numpy array or torch tensor."""
    if x is None:
        return None, None, False
    if _is_cuda_tensor(x):
        torch = _torch()
        want = {np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            x = x.to(want).contiguous()
        return x.data_ptr(), x, True
    if hasattr(x, "numpy"):
        x = x.numpy()
    a = np.ascontiguousarray(np.asarray(x), dtype=dtype)
    return a.ctypes.data, a, False


def default_options(**overrides) -> Options:
    o = Options()
    lib().kcore_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def default_serve_options(sweep: Options | None = None, **overrides) -> ServeOptions:
    o = ServeOptions()
    lib().kcore_default_serve_options(ctypes.byref(o))
    if sweep is not None:
        o.sweep = sweep
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown serve option {k}")
        setattr(o, k, v)
    return o


class Graph:
    """A cleaned graph resident on the GPU (kcore_create / kcore_create_coo)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        n, nnz, rp = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        check(lib().kcore_graph_info(self._h, ctypes.byref(n), ctypes.byref(nnz),
                                     ctypes.byref(rp)), "kcore_graph_info")
        self.n, self.nnz, self.row_ptr_bytes = n.value, nnz.value, rp.value

    # ---------------------------------------------------------------- create
    @classmethod
    def from_coo(cls, n: int, src, dst, row_ptr_bytes: int = 4, options: Options | None = None,
                 stream=None) -> "Graph":
        ps, ks, ds = _ptr(src, np.int32)
        pd, kd, dd = _ptr(dst, np.int32)
        if ds != dd:
            raise ValueError("src and dst must both be host arrays or both CUDA tensors")
        nnz = int(ks.shape[0]) if hasattr(ks, "shape") else int(ks.numel())
        h = ctypes.c_void_p()
        flags = KCORE_IN_DEVICE if ds else 0
        check(lib().kcore_create_coo(n, nnz, ps, pd, row_ptr_bytes, flags,
                                     ctypes.byref(options) if options else None,
                                     _stream(stream), ctypes.byref(h)), "kcore_create_coo")
        return cls(h.value)

    @classmethod
    def from_csr(cls, n: int, row_ptr, col_idx, clean: bool = False,
                 options: Options | None = None, stream=None) -> "Graph":
        rp_dtype = np.int64 if str(getattr(row_ptr, "dtype", "")).endswith("int64") else np.int32
        pr, kr, dr = _ptr(row_ptr, rp_dtype)
        pc, kc, dc = _ptr(col_idx, np.int32)
        flags = (KCORE_IN_DEVICE if dr else 0) | (KCORE_IN_CLEAN if clean else 0)
        h = ctypes.c_void_p()
        check(lib().kcore_create(n, pr, 8 if rp_dtype == np.int64 else 4, pc, flags,
                                 ctypes.byref(options) if options else None, _stream(stream),
                                 ctypes.byref(h)), "kcore_create")
        return cls(h.value)

    # ---------------------------------------------------------------- run
    def run(self, out=None, device: bool = True, sync_mode: bool = False, refined: bool | None = None,
            wait: bool = True, stream=None, check_status: bool = True, graph: bool = False):
        """Coreness of every vertex.  Returns `out` (allocated when None: an
        int32 CUDA tensor if device else a numpy array).  `refined`: activation
        rule; None = the library default (refined when asynchronous, the
        simple rule of Alg. 3 when synchronous)."""
        if refined is None:
            refined = not sync_mode
        if out is None:
            if device:
                torch = _torch()
                out = torch.empty(self.n, dtype=torch.int32, device="cuda")
            else:
                out = np.empty(self.n, dtype=np.int32)
        is_dev = _is_cuda_tensor(out)
        ptr = out.data_ptr() if is_dev else out.ctypes.data
        flags = (KCORE_OUT_DEVICE if is_dev else 0) | (KCORE_SYNC_MODE if sync_mode else 0) | \
            (KCORE_REFINED if refined and sync_mode else 0) | \
            (KCORE_SIMPLE if not refined and not sync_mode else 0) | (0 if wait else KCORE_ASYNC) | \
            (KCORE_GRAPH if graph else 0)
        st = lib().kcore_run(self._h, ptr, flags, _stream(stream))
        if check_status:
            check(st, "kcore_run")
        self.last_status = st
        return out

    def run_from(self, start, frontier=None, out=None, device: bool = True, sync_mode: bool = False,
                 refined: bool | None = None, wait: bool = True, stream=None, check_status: bool = True):
        """The iteration started from upper bounds `start` (n values >= the
        coreness) with only `frontier` active (None: every vertex): dynamic
        maintenance after edge deletions (old coreness, endpoints active) or
        insertions (old coreness + number inserted, everything active).
        `start` and `frontier` are both numpy arrays or both CUDA tensors."""
        if refined is None:
            refined = not sync_mode
        ps, ks, ds = _ptr(start, np.int32)
        pf, kf, df, nf = None, None, ds, 0
        if frontier is not None:
            pf, kf, df = _ptr(frontier, np.int32)
            nf = int(kf.shape[0]) if hasattr(kf, "shape") else int(kf.numel())
        if ds != df:
            raise ValueError("start and frontier must both be host arrays or both CUDA tensors")
        if out is None:
            if device:
                torch = _torch()
                out = torch.empty(self.n, dtype=torch.int32, device="cuda")
            else:
                out = np.empty(self.n, dtype=np.int32)
        is_dev = _is_cuda_tensor(out)
        optr = out.data_ptr() if is_dev else out.ctypes.data
        flags = (KCORE_IN_DEVICE if ds else 0) | (KCORE_OUT_DEVICE if is_dev else 0) | \
            (KCORE_SYNC_MODE if sync_mode else 0) | (KCORE_REFINED if refined and sync_mode else 0) | \
            (KCORE_SIMPLE if not refined and not sync_mode else 0) | (0 if wait else KCORE_ASYNC)
        st = lib().kcore_run_from(self._h, ps, pf, nf, optr, flags, _stream(stream))
        if check_status:
            check(st, "kcore_run_from")
        self.last_status = st
        return out

    def wait(self) -> int:
        return lib().kcore_wait(self._h)

    def set_options(self, options: Options, stream=None) -> None:
        check(lib().kcore_set_options(self._h, ctypes.byref(options), _stream(stream)),
              "kcore_set_options")

    def stats(self) -> dict:
        s = RunStats()
        check(lib().kcore_stats(self._h, ctypes.byref(s)), "kcore_stats")
        return {k: getattr(s, k) for k, _ in RunStats._fields_}

    def trace(self, cap: int = 1 << 16, with_time: bool = False):
        """Per-sweep (frontier size, frontier degree sum, updates[, start ns])."""
        f = np.zeros(cap, np.int64)
        d = np.zeros(cap, np.int64)
        u = np.zeros(cap, np.int64)
        t = np.zeros(cap, np.int64)
        cnt = ctypes.c_int64()
        check(lib().kcore_sweep_trace(self._h, f.ctypes.data, d.ctypes.data, u.ctypes.data,
                                      t.ctypes.data, cap, ctypes.byref(cnt)), "kcore_sweep_trace")
        k = cnt.value
        if with_time:
            return f[:k], d[:k], u[:k], t[:k]
        return f[:k], d[:k], u[:k]

    def trace_detail(self, cap: int = 1 << 16):
        """Per-sweep (adjacency entries read, sum of estimate decreases)."""
        r = np.zeros(cap, np.int64)
        dec = np.zeros(cap, np.int64)
        cnt = ctypes.c_int64()
        check(lib().kcore_sweep_detail(self._h, r.ctypes.data, dec.ctypes.data, cap,
                                       ctypes.byref(cnt)), "kcore_sweep_detail")
        return r[:cnt.value], dec[:cnt.value]

    def trace_tiers(self, cap: int = 1 << 16):
        """Per-sweep frontier size and degree sum per degree tier: two arrays of
        shape (sweeps, 3), tiers thread / warp / CTA."""
        f = np.zeros(3 * cap, np.int64)
        d = np.zeros(3 * cap, np.int64)
        cnt = ctypes.c_int64()
        check(lib().kcore_sweep_tiers(self._h, f.ctypes.data, d.ctypes.data, cap,
                                      ctypes.byref(cnt)), "kcore_sweep_tiers")
        k = cnt.value
        return f[:3 * k].reshape(k, 3), d[:3 * k].reshape(k, 3)

    def row_ptr_host(self):
        """row_ptr of the cleaned graph as a numpy array."""
        rp = np.empty(self.n + 1, dtype=np.int64 if self.row_ptr_bytes == 8 else np.int32)
        check(lib().kcore_copy_csr(self._h, rp.ctypes.data, None, 0), "kcore_copy_csr")
        return rp

    def csr(self):
        """(row_ptr, col_idx) of the cleaned graph, as numpy arrays."""
        rp = np.empty(self.n + 1, dtype=np.int64 if self.row_ptr_bytes == 8 else np.int32)
        col = np.empty(max(self.nnz, 1), dtype=np.int32)
        check(lib().kcore_copy_csr(self._h, rp.ctypes.data, col.ctypes.data, 0), "kcore_copy_csr")
        return rp, col[: self.nnz]

    def close(self) -> None:
        if self._h and self._h.value:
            lib().kcore_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchEngine:
    """Continuous-batching engine (kcore_batch_*): submit graphs, poll results."""

    def __init__(self, options: ServeOptions | None = None):
        h = ctypes.c_void_p()
        check(lib().kcore_batch_create(ctypes.byref(options) if options else None,
                                       ctypes.byref(h)), "kcore_batch_create")
        self._h = h

    def submit_coo(self, n: int, src, dst) -> int:
        ps, ks, _ = _ptr(src, np.int32)
        pd, kd, _ = _ptr(dst, np.int32)
        t = ctypes.c_uint64()
        check(lib().kcore_submit_coo(self._h, n, int(ks.shape[0]), ps, pd, 0, ctypes.byref(t)),
              "kcore_submit_coo")
        return t.value

    def submit_csr(self, n: int, row_ptr, col_idx, clean: bool = False) -> int:
        rp_dtype = np.int64 if str(getattr(row_ptr, "dtype", "")).endswith("int64") else np.int32
        pr, kr, _ = _ptr(row_ptr, rp_dtype)
        pc, kc, _ = _ptr(col_idx, np.int32)
        t = ctypes.c_uint64()
        check(lib().kcore_submit(self._h, n, pr, 8 if rp_dtype == np.int64 else 4, pc,
                                 KCORE_IN_CLEAN if clean else 0, ctypes.byref(t)), "kcore_submit")
        return t.value

    def poll(self, ticket: int, n: int | None = None, timeout_us: int = -1):
        """(status, coreness or None).  status is KCORE_OK, KCORE_PENDING or an error."""
        out = np.empty(max(n or 0, 1), dtype=np.int32) if n is not None else None
        st = lib().kcore_poll(self._h, ticket, out.ctypes.data if out is not None else None,
                              timeout_us)
        if st == KCORE_OK:
            return st, (out[:n] if out is not None else None)
        return st, None

    def poll_info(self, ticket: int, n: int | None = None, timeout_us: int = -1):
        """(status, coreness or None, info dict or None): kcore_poll_info.  The
        info (times on the monotonic clock of time.perf_counter, launch
        numbers) is filled on every return but KCORE_PENDING."""
        out = np.empty(max(n or 0, 1), dtype=np.int32) if n is not None else None
        info = TicketInfo()
        st = lib().kcore_poll_info(self._h, ticket, out.ctypes.data if out is not None else None,
                                   timeout_us, ctypes.byref(info))
        if st == KCORE_PENDING:
            return st, None, None
        d = {k: getattr(info, k) for k, _ in TicketInfo._fields_}
        return st, (out[:n] if (st == KCORE_OK and out is not None) else None), d

    def cancel(self, ticket: int) -> int:
        return lib().kcore_cancel(self._h, ticket)

    def step(self) -> int:
        a = ctypes.c_int64()
        check(lib().kcore_batch_step(self._h, ctypes.byref(a)), "kcore_batch_step")
        return a.value

    def stats(self) -> dict:
        s = BatchStats()
        check(lib().kcore_batch_stats_get(self._h, ctypes.byref(s)), "kcore_batch_stats_get")
        return {k: getattr(s, k) for k, _ in BatchStats._fields_}

    def close(self) -> None:
        if self._h and self._h.value:
            lib().kcore_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
