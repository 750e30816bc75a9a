"""Seeded synthetic graph inputs shared by the GPU library's tests/bench and the oracle.

This module only generates raw directed edge samples ``(src, dst)`` (int32 numpy
arrays) plus the vertex count.  It contains none of the k-core method: no
symmetrisation, deduplication, degrees or coreness.  The C source
``graphgen.c`` is compiled on first use with the host ``gcc``.

The workloads stand in for the paper's SNAP road, web and social graphs
(Table I), which are not available here; see ``WORKLOADS``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import tempfile
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "_libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into _libgraphgen.so (skipped when up to date)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError as e:
        os.unlink(tmp)
        raise RuntimeError(f"graphgen build failed:\n{e.stderr}") from e
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, u64, p32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        dbl, cint = ctypes.c_double, ctypes.c_int
        lib.gg_er.argtypes = [i64, i64, u64, p32, p32]
        lib.gg_er.restype = i64
        lib.gg_damaged_grid.argtypes = [i64, dbl, dbl, u64, p32, p32]
        lib.gg_damaged_grid.restype = i64
        lib.gg_rmat.argtypes = [i64, i64, dbl, dbl, dbl, cint, u64, p32, p32]
        lib.gg_rmat.restype = i64
        lib.gg_planted.argtypes = [i64, i64, dbl, u64, p32, p32]
        lib.gg_planted.restype = i64
        lib.gg_stream_params.argtypes = [u64, i64, i64, i64, ctypes.POINTER(i64),
                                         ctypes.POINTER(ctypes.c_int32)]
        lib.gg_stream_params.restype = None
        lib.gg_random.argtypes = [u64, u64, u64]
        lib.gg_random.restype = u64
        _lib = lib
    return _lib


@dataclass
class EdgeList:
    """Raw directed edge samples on vertices [0, n)."""
    n: int
    src: np.ndarray
    dst: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def samples(self) -> int:
        return int(self.src.shape[0])


def _buf(cap: int):
    return np.empty(max(cap, 1), dtype=np.int32), np.empty(max(cap, 1), dtype=np.int32)


def er(n: int, m: int, seed: int = 0) -> EdgeList:
    """G(n, m): m distinct uniform non-loop pairs (each listed once)."""
    s, d = _buf(m)
    got = _load().gg_er(n, m, seed, s.ctypes.data, d.ctypes.data)
    if got < 0:
        raise ValueError(f"er({n}, {m}) impossible")
    return EdgeList(n, s[:got], d[:got], f"er_n{n}_m{m}_s{seed}",
                    {"family": "er", "m": m, "seed": seed})


def damaged_grid(L: int, p_del: float = 0.30, p_diag: float = 0.05, seed: int = 0) -> EdgeList:
    """L x L 4-neighbour grid, edges deleted w.p. p_del, plus random diagonals."""
    cap = 2 * L * (L - 1) + L * L
    s, d = _buf(cap)
    got = _load().gg_damaged_grid(L, p_del, p_diag, seed, s.ctypes.data, d.ctypes.data)
    if got < 0:
        raise ValueError("bad grid size")
    return EdgeList(L * L, s[:got].copy(), d[:got].copy(), f"grid_L{L}_s{seed}",
                    {"family": "grid", "L": L, "p_del": p_del, "p_diag": p_diag, "seed": seed})


def rmat(n: int, samples: int, a: float, b: float, c: float, seed: int = 0,
         relabel: bool = True) -> EdgeList:
    """R-MAT samples on n vertices (scale = ceil(log2 n), out-of-range redrawn)."""
    s, d = _buf(samples)
    got = _load().gg_rmat(n, samples, a, b, c, int(relabel), seed, s.ctypes.data, d.ctypes.data)
    if got < 0:
        raise ValueError("bad rmat parameters")
    return EdgeList(n, s[:got], d[:got], f"rmat_n{n}_e{samples}_s{seed}",
                    {"family": "rmat", "abc": (a, b, c), "relabel": relabel, "seed": seed})


def planted(n: int, k: int, p: float, seed: int = 0) -> EdgeList:
    """G(k, p) on k vertices chosen uniformly from [0, n)."""
    cap = k * (k - 1) // 2
    s, d = _buf(cap)
    got = _load().gg_planted(n, k, p, seed, s.ctypes.data, d.ctypes.data)
    if got < 0:
        raise ValueError("bad planted parameters")
    return EdgeList(n, s[:got].copy(), d[:got].copy(), f"planted_n{n}_k{k}_s{seed}",
                    {"family": "planted", "k": k, "p": p, "seed": seed})


def union(*parts: EdgeList, name: str = "") -> EdgeList:
    """Concatenate edge samples of graphs on the same vertex set."""
    n = max(p.n for p in parts)
    return EdgeList(n, np.concatenate([p.src for p in parts]),
                    np.concatenate([p.dst for p in parts]), name,
                    {"parts": [p.name for p in parts]})


# ---------------------------------------------------------------- batch stream
STREAM_NMIN, STREAM_NMAX = 100, 200_000
STREAM_FAMILIES = ("er", "rmat", "grid")


def stream_params(index: int, seed: int = 0, nmin: int = STREAM_NMIN,
                  nmax: int = STREAM_NMAX) -> tuple[int, str]:
    n = ctypes.c_int64()
    fam = ctypes.c_int32()
    _load().gg_stream_params(seed, index, nmin, nmax, ctypes.byref(n), ctypes.byref(fam))
    return int(n.value), STREAM_FAMILIES[fam.value]


def stream_graph(index: int, seed: int = 0, nmin: int = STREAM_NMIN,
                 nmax: int = STREAM_NMAX) -> EdgeList:
    """Graph `index` of the batch stream; its own seed is the index."""
    n, fam = stream_params(index, seed, nmin, nmax)
    if fam == "er":
        g = er(n, min(4 * n, n * (n - 1) // 2), seed=index)
    elif fam == "rmat":
        g = rmat(n, 8 * n, 0.57, 0.19, 0.19, seed=index, relabel=True)
    else:
        g = damaged_grid(int(round(n ** 0.5)), seed=index)
    g.name = f"stream{index}_{fam}_n{g.n}"
    g.meta["family"] = fam
    return g


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative Exp(rate) gaps."""
    lib = _load()
    u = np.array([lib.gg_random(seed, 0xA77, i) for i in range(count)], dtype=np.uint64)
    unit = (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    gaps = -np.log1p(-unit) / rate_per_s
    return np.cumsum(gaps)


# ---------------------------------------------------------------- named workloads
def _w_er10k():
    g = er(10_000, 50_000, seed=0)
    g.name = "er_n10000_m50000"
    return g


def _w_road2048():
    g = damaged_grid(2048, 0.30, 0.05, seed=0)
    g.name = "road_grid2048_del30_diag5"
    return g


def _w_rmat22():
    n = 1 << 22
    g = rmat(n, 16 * n, 0.57, 0.19, 0.19, seed=0, relabel=True)
    g.name = "rmat22_ef16"
    return g


def _w_rmat24_planted():
    n = 1 << 24
    base = rmat(n, 32 * n, 0.45, 0.22, 0.22, seed=0, relabel=True)
    core = planted(n, 5000, 0.5, seed=1)
    return union(base, core, name="rmat24_ef32_planted5000")


WORKLOADS = {
    # name: (builder, row_ptr bytes)
    "er10k": (_w_er10k, 4),
    "road2048": (_w_road2048, 4),
    "rmat22": (_w_rmat22, 8),
    "rmat24_planted": (_w_rmat24_planted, 8),
}


def workload(name: str) -> EdgeList:
    builder, rp = WORKLOADS[name]
    g = builder()
    g.meta["row_ptr_bytes"] = rp
    return g


if __name__ == "__main__":  # pragma: no cover
    for nm in sys.argv[1:] or ["er10k"]:
        g = workload(nm)
        print(nm, g.n, g.samples)
