"""The synthetic inputs against the recipe they follow (the stand-ins for the
paper's SNAP graphs and the serving stream): counts, structure and the
distributions the generators promise, with tolerances of four binomial
standard deviations, and determinism by seed."""
import math

import numpy as np
import pytest

import graphgen
import oracle


def pairs(g):
    a = np.minimum(g.src, g.dst).astype(np.int64)
    b = np.maximum(g.src, g.dst).astype(np.int64)
    return a * g.n + b


def test_er_distinct_non_loop_pairs_and_seeded():
    g = graphgen.er(1000, 5000, seed=3)
    assert g.samples == 5000 and (g.src != g.dst).all()
    assert g.src.min() >= 0 and max(g.src.max(), g.dst.max()) < 1000
    assert np.unique(pairs(g)).size == 5000
    h = graphgen.er(1000, 5000, seed=3)
    assert (h.src == g.src).all() and (h.dst == g.dst).all()
    assert not (graphgen.er(1000, 5000, seed=4).src == g.src).all()
    with pytest.raises(ValueError):
        graphgen.er(4, 7)                       # more than n(n-1)/2 edges


def test_damaged_grid_structure_and_rates():
    L = 128
    g = graphgen.damaged_grid(L, 0.30, 0.05, seed=2)
    assert g.n == L * L and (g.src != g.dst).all()
    dx = np.abs(g.src % L - g.dst % L)
    dy = np.abs(g.src // L - g.dst // L)
    grid = ((dx == 1) & (dy == 0)) | ((dx == 0) & (dy == 1))
    diag = (dx == 1) & (dy == 1)
    assert (grid | diag).all()                  # only grid edges and diagonals
    full = 2 * L * (L - 1)
    kept = int(grid.sum())
    assert np.unique(pairs(graphgen.EdgeList(g.n, g.src[grid], g.dst[grid], "", {}))).size == kept
    assert abs(kept - 0.7 * full) < 4 * math.sqrt(full * 0.3 * 0.7)
    nd = int(diag.sum())
    assert abs(nd - 0.05 * g.n) < 4 * math.sqrt(g.n * 0.05 * 0.95)


def test_road2048_workload_matches_its_stated_sizes():
    g = graphgen.workload("road2048")
    rp, col = oracle.csr_build(g.n, g.src, g.dst)
    m = int(rp[-1]) // 2
    assert g.n == 4_194_304 and m == 6_076_673
    assert round(2 * m / g.n, 2) == 2.90
    assert int(oracle.coreness(g.n, rp, col).max()) == 3


def test_rmat_quadrants_and_range():
    n, S = 1 << 16, 1 << 20
    g = graphgen.rmat(n, S, 0.57, 0.19, 0.19, seed=5, relabel=False)
    assert g.samples == S and g.src.min() >= 0 and max(g.src.max(), g.dst.max()) < n
    hs, hd = g.src >> 15, g.dst >> 15           # top level of the recursion
    tol = 4 * math.sqrt(0.25 / S)
    for (qs, qd), p in {(0, 0): 0.57, (0, 1): 0.19, (1, 0): 0.19, (1, 1): 0.05}.items():
        assert abs(float(((hs == qs) & (hd == qd)).mean()) - p) < tol, (qs, qd)
    r = graphgen.rmat(n, S, 0.57, 0.19, 0.19, seed=5, relabel=True)
    assert abs(float(((r.src >> 15) == 0).mean()) - 0.5) < 0.05   # labels permuted
    deg = np.bincount(np.concatenate([r.src, r.dst]), minlength=n)
    assert deg.max() > 50 * deg.mean()          # heavy-tailed degrees
    odd = graphgen.rmat(1000, 10_000, 0.57, 0.19, 0.19, seed=1)   # n not a power of two
    assert odd.samples == 10_000 and max(odd.src.max(), odd.dst.max()) < 1000


def test_planted_core():
    g = graphgen.planted(10_000, 200, 0.5, seed=1)
    assert np.unique(np.concatenate([g.src, g.dst])).size == 200
    assert (g.src != g.dst).all() and np.unique(pairs(g)).size == g.samples
    pairs_all = 200 * 199 // 2
    assert abs(g.samples - 0.5 * pairs_all) < 4 * math.sqrt(pairs_all * 0.25)


def test_stream_sizes_families_and_arrivals():
    N = 20_000
    params = [graphgen.stream_params(i) for i in range(N)]
    ns = np.array([p[0] for p in params], dtype=np.float64)
    assert ns.min() >= 100 and ns.max() <= 200_000
    lo, hi = math.log(100), math.log(200_000)
    sd = (hi - lo) / math.sqrt(12) / math.sqrt(N)
    assert abs(float(np.log(ns).mean()) - (lo + hi) / 2) < 4 * sd        # log-uniform
    for fam in graphgen.STREAM_FAMILIES:
        share = sum(1 for p in params if p[1] == fam) / N
        assert abs(share - 1 / 3) < 4 * math.sqrt(2 / 9 / N), fam
    for i in range(6):                          # sample counts per family
        g = graphgen.stream_graph(i)
        n, fam = graphgen.stream_params(i)
        if fam == "er":
            assert g.samples == min(4 * n, n * (n - 1) // 2)
        elif fam == "rmat":
            assert g.samples == 8 * n and g.n == n
        else:
            assert g.n == round(n ** 0.5) ** 2
    t = graphgen.poisson_arrivals(N, 1000.0, seed=1)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(float(gaps.mean()) - 1e-3) < 4 * 1e-3 / math.sqrt(N)
    assert abs(float(gaps.std() / gaps.mean()) - 1.0) < 0.05              # exponential gaps
    assert (graphgen.poisson_arrivals(100, 1000.0, seed=1) == t[:100]).all()
