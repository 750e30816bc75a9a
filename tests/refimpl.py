"""Independent brute-force references used only to pin the oracle.

Nothing here is shared with ``oracle/`` or the CUDA library: each function is
a second, deliberately different statement of a definition, so that a slip in
the oracle (a dropped term, a wrong index, a wrong start value) shows up as a
disagreement.

* ``coreness_subsets``  -- Def. 1 literally: core(v) is the largest k such that
  some vertex set S containing v induces a subgraph of minimum degree >= k
  (the k-core is the union of all such S).  Exponential; n <= ~14.
* ``coreness_peel_levels`` -- repeated deletion: for k = 1, 2, ..., delete
  vertices whose remaining degree is < k until none is left to delete; a vertex
  first deleted at level k has coreness k - 1.  Vectorised with numpy so it
  also runs on graphs with millions of vertices.
* ``hindex_sorted``     -- h-index from the sorted list: the largest i such that
  the i-th largest value is >= i, capped.
* ``csr_scipy``         -- the cleaned CSR via scipy.sparse (library routine).
"""
from __future__ import annotations

import itertools

import numpy as np


def adjacency_masks(n: int, edges) -> list[int]:
    adj = [0] * n
    for a, b in edges:
        if a != b:
            adj[a] |= 1 << b
            adj[b] |= 1 << a
    return adj


def coreness_subsets(n: int, edges) -> list[int]:
    adj = adjacency_masks(n, edges)
    core = [0] * n
    for S in range(1, 1 << n):
        md = None
        members = [v for v in range(n) if S >> v & 1]
        for v in members:
            d = bin(adj[v] & S).count("1")
            md = d if md is None or d < md else md
        for v in members:
            if md > core[v]:
                core[v] = md
    return core


def coreness_peel_levels(n: int, row_ptr, col) -> np.ndarray:
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    alive = np.ones(n, dtype=bool)
    core = np.zeros(n, dtype=np.int64)
    k = 0
    while alive.any():
        k += 1
        while True:
            live_edge = alive[rows] & alive[col]
            d = np.bincount(rows[live_edge], minlength=n)
            drop = alive & (d < k)
            if not drop.any():
                break
            core[drop] = k - 1
            alive &= ~drop
    return core.astype(np.int32)


def hindex_sorted(values, cap: int) -> int:
    s = sorted((int(x) for x in values), reverse=True)
    h = 0
    for i, x in enumerate(s, start=1):
        if x >= i:
            h = i
    return min(h, cap)


def hindex_uncapped_rows(n: int, row_ptr, col, vals) -> np.ndarray:
    """Per-vertex h-index of the neighbours' vals, vectorised by sorting each
    row's values in descending order (numpy lexsort)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    deg = np.diff(row_ptr)
    rows = np.repeat(np.arange(n, dtype=np.int64), deg)
    x = np.asarray(vals, dtype=np.int64)[col]
    order = np.lexsort((-x, rows))          # by row, then value descending
    xs = x[order]
    rank = np.arange(col.shape[0], dtype=np.int64) - row_ptr[rows[order]] + 1
    ok = xs >= rank
    h = np.zeros(n, dtype=np.int64)
    np.maximum.at(h, rows[order][ok], rank[ok])
    return h.astype(np.int32)


def csr_scipy(n: int, src, dst):
    import scipy.sparse as sp
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    s, d = src[keep], dst[keep]
    a = sp.coo_matrix((np.ones(s.shape[0], dtype=np.int8), (s, d)), shape=(n, n)).tocsr()
    a = (a + a.T).tocsr()
    a.sum_duplicates()
    a.sort_indices()
    return a.indptr.astype(np.int64), a.indices.astype(np.int32)


def all_graphs(n: int):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield [p for i, p in enumerate(pairs) if mask >> i & 1]
