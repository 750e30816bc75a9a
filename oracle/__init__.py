"""k-core ORACLE (test infrastructure).

Plain CPU reference for what the GPU library computes.  Only the tests, the
``__graft_entry__.smoke()`` check and the benchmark's CPU-baseline leg may use
it; the library itself never imports it and has no CPU fallback.  It shares no
code with the CUDA path: ``kcore_oracle.c`` is compiled here with ``gcc``.

Functions and the passages they follow:
  * ``csr_build``      -- undirected simple CSR with sorted rows (Sec. IV-A:
    undirected, self-loops removed; Sec. III-B: sorted neighbour vectors).
  * ``hindex``         -- capped h-index, the reading of computeCoreness in
    Alg. 1 (its body is not given in the paper).
  * ``coreness``       -- Batagelj-Zaversnik peeling (Sec. II), i.e. the
    coreness of Def. 1.
  * ``montresor_sync`` -- synchronous rounds of Alg. 3 with the selective
    activation rule of Sec. III-B (optionally the refined rule of Sec. IV).

Every function here is pinned by tests/test_oracle.py against brute force from
Def. 1, closed forms, invariants and library routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kcore_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_libkcore_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile kcore_oracle.c (plain C, -O2, single-threaded)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError as e:
        os.unlink(tmp)
        raise RuntimeError(f"oracle build failed:\n{e.stderr}") from e
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, vp = ctypes.c_int64, ctypes.c_void_p
        lib.orc_csr_build.argtypes = [i64, i64, vp, vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
        lib.orc_csr_build.restype = i64
        lib.orc_free.argtypes = [vp]
        lib.orc_free.restype = None
        lib.orc_hindex.argtypes = [vp, i64, ctypes.c_int32]
        lib.orc_hindex.restype = ctypes.c_int32
        lib.orc_bz.argtypes = [i64, vp, vp, vp]
        lib.orc_bz.restype = ctypes.c_int
        lib.orc_montresor_sync.argtypes = [i64, vp, vp, i64, ctypes.c_int, vp, vp, vp, i64]
        lib.orc_montresor_sync.restype = i64
        _lib = lib
    return _lib


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int64)


def csr_build(n: int, src, dst) -> tuple[np.ndarray, np.ndarray]:
    """Raw edge samples -> (row_ptr int64[n+1], col int32[2m]) of the simple
    undirected graph, rows ascending."""
    lib = _load()
    s, d = _i32(src), _i32(dst)
    if s.shape != d.shape:
        raise ValueError("src/dst length mismatch")
    rp, cp = ctypes.c_void_p(), ctypes.c_void_p()
    nnz = lib.orc_csr_build(n, s.shape[0], s.ctypes.data, d.ctypes.data,
                            ctypes.byref(rp), ctypes.byref(cp))
    if nnz < 0:
        raise ValueError("orc_csr_build: invalid input or out of memory")
    try:
        row_ptr = np.ctypeslib.as_array(ctypes.cast(rp, ctypes.POINTER(ctypes.c_int64)),
                                        shape=(n + 1,)).copy()
        col = (np.ctypeslib.as_array(ctypes.cast(cp, ctypes.POINTER(ctypes.c_int32)),
                                     shape=(nnz,)).copy() if nnz else np.zeros(0, np.int32))
    finally:
        lib.orc_free(rp)
        lib.orc_free(cp)
    return row_ptr, col


def hindex(values, cap: int) -> int:
    """Largest h <= cap with at least h of `values` >= h."""
    v = _i32(values)
    r = _load().orc_hindex(v.ctypes.data, v.shape[0], int(cap))
    if r < 0:
        raise ValueError("bad h-index input")
    return int(r)


def coreness(n: int, row_ptr, col) -> np.ndarray:
    """Coreness of every vertex of a clean undirected CSR (Batagelj-Zaversnik)."""
    rp, c = _i64(row_ptr), _i32(col)
    out = np.zeros(n, dtype=np.int32)
    if _load().orc_bz(n, rp.ctypes.data, c.ctypes.data, out.ctypes.data) != 0:
        raise MemoryError("orc_bz")
    return out


def montresor_sync(n: int, row_ptr, col, max_rounds: int = 1 << 40, refined: bool = False,
                   record: int = 0):
    """Synchronous rounds (Alg. 3).  Returns (rounds or -1, est, frontier[:record],
    changed[:record])."""
    rp, c = _i64(row_ptr), _i32(col)
    est = np.zeros(max(n, 1), dtype=np.int32)
    fr = np.zeros(max(record, 1), dtype=np.int64)
    ch = np.zeros(max(record, 1), dtype=np.int64)
    r = _load().orc_montresor_sync(n, rp.ctypes.data, c.ctypes.data, int(max_rounds),
                                   int(refined), est.ctypes.data,
                                   fr.ctypes.data if record else None,
                                   ch.ctypes.data if record else None, int(record))
    if r == -2:
        raise MemoryError("orc_montresor_sync")
    used = min(record, r if r >= 0 else int(max_rounds))
    return int(r), est[:n], fr[:used], ch[:used]


def from_edges(g) -> tuple[np.ndarray, np.ndarray]:
    """CSR of a graphgen.EdgeList (convenience for tests/bench)."""
    return csr_build(g.n, g.src, g.dst)
