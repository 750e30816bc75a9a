"""Pins for the CPU oracle (CPU only).

The oracle is checked against things other than itself: Def. 1 by brute force
over vertex subsets (exhaustively on every labelled graph with n <= 6),
repeated min-degree deletion, closed forms, hand-derived fixtures, invariants,
scipy's CSR construction, networkx, and a sort-based h-index.
"""
import numpy as np
import pytest

import graphgen
import oracle
from tests import golden_io, refimpl


def csr_of(n, edges):
    e = np.array(edges, dtype=np.int32).reshape(-1, 2)
    return oracle.csr_build(n, e[:, 0], e[:, 1])


def bz_of(n, edges):
    rp, col = csr_of(n, edges)
    return oracle.coreness(n, rp, col)


# ------------------------------------------------------------------ Def. 1 brute force
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_bz_equals_def1_exhaustive_small(n):
    for edges in refimpl.all_graphs(n):
        assert bz_of(n, edges).tolist() == refimpl.coreness_subsets(n, edges), edges


def test_bz_equals_def1_exhaustive_n6():
    n = 6
    for edges in refimpl.all_graphs(n):
        assert bz_of(n, edges).tolist() == refimpl.coreness_subsets(n, edges), edges


def test_bz_equals_def1_random_n12():
    rng = np.random.default_rng(7)
    for trial in range(40):
        n = 12
        p = rng.uniform(0.1, 0.7)
        edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
        assert bz_of(n, edges).tolist() == refimpl.coreness_subsets(n, edges)


def test_bz_equals_repeated_deletion_random():
    rng = np.random.default_rng(11)
    for trial in range(60):
        n = int(rng.integers(1, 200))
        m = int(rng.integers(0, 4 * n + 1))
        src = rng.integers(0, n, m).astype(np.int32)
        dst = rng.integers(0, n, m).astype(np.int32)
        rp, col = oracle.csr_build(n, src, dst)
        np.testing.assert_array_equal(oracle.coreness(n, rp, col),
                                      refimpl.coreness_peel_levels(n, rp, col))


# ------------------------------------------------------------------ closed forms
def complete(n):
    return [(a, b) for a in range(n) for b in range(a + 1, n)]


def cycle(n):
    return [(i, (i + 1) % n) for i in range(n)]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 40])
def test_complete_graph(n):
    assert (bz_of(n, complete(n)) == n - 1).all()


@pytest.mark.parametrize("n", [3, 4, 10, 101])
def test_cycle(n):
    assert (bz_of(n, cycle(n)) == 2).all()


def test_path_star_tree_isolated():
    assert (bz_of(50, [(i, i + 1) for i in range(49)]) == 1).all()
    assert (bz_of(30, [(0, i) for i in range(1, 30)]) == 1).all()
    rng = np.random.default_rng(3)
    n = 300
    tree = [(i, int(rng.integers(0, i))) for i in range(1, n)]
    assert (bz_of(n, tree) == 1).all()
    assert (bz_of(5, []) == 0).all()


@pytest.mark.parametrize("a,b", [(1, 1), (2, 5), (4, 4), (3, 9)])
def test_complete_bipartite(a, b):
    edges = [(i, a + j) for i in range(a) for j in range(b)]
    assert (bz_of(a + b, edges) == min(a, b)).all()


@pytest.mark.parametrize("n,r", [(20, 4), (31, 6), (64, 10)])
def test_regular_circulant(n, r):
    edges = [(i, (i + s) % n) for i in range(n) for s in range(1, r // 2 + 1)]
    assert (bz_of(n, edges) == r).all()


def test_full_grid_is_2():
    L = 40
    g = graphgen.damaged_grid(L, p_del=0.0, p_diag=0.0)
    rp, col = oracle.csr_build(g.n, g.src, g.dst)
    assert (oracle.coreness(g.n, rp, col) == 2).all()


def test_disjoint_union_is_per_component():
    parts = [(6, complete(6)), (9, cycle(9)), (4, [(0, 1), (1, 2)]), (1, [])]
    edges, off, expect = [], 0, []
    for n, e in parts:
        edges += [(a + off, b + off) for a, b in e]
        expect += bz_of(n, e).tolist()
        off += n
    assert bz_of(off, edges).tolist() == expect


# ------------------------------------------------------------------ fixtures
@pytest.mark.parametrize("fx", golden_io.all_fixtures(), ids=lambda f: f["name"])
def test_golden_fixture(fx):
    rp, col = oracle.csr_build(fx["n"], fx["src"], fx["dst"])
    assert oracle.coreness(fx["n"], rp, col).tolist() == fx["coreness"]
    if "row_ptr" in fx:
        assert rp.tolist() == fx["row_ptr"]
        assert col.tolist() == fx["col"]


# ------------------------------------------------------------------ CSR build
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_csr_build_matches_scipy(seed):
    rng = np.random.default_rng(seed)
    n = 500
    m = 4000
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    src[:50] = dst[:50]                      # self-loops
    src[50:100], dst[50:100] = dst[100:150], src[100:150]   # reversed repeats
    rp, col = oracle.csr_build(n, src, dst)
    rp2, col2 = refimpl.csr_scipy(n, src, dst)
    np.testing.assert_array_equal(rp, rp2)
    np.testing.assert_array_equal(col, col2)


def test_csr_build_workload_matches_scipy():
    g = graphgen.rmat(1 << 14, 16 << 14, 0.57, 0.19, 0.19, seed=5)
    rp, col = oracle.csr_build(g.n, g.src, g.dst)
    rp2, col2 = refimpl.csr_scipy(g.n, g.src, g.dst)
    np.testing.assert_array_equal(rp, rp2)
    np.testing.assert_array_equal(col, col2)


def test_csr_build_rejects_out_of_range():
    with pytest.raises(ValueError):
        oracle.csr_build(3, np.array([0, 3], np.int32), np.array([1, 1], np.int32))


# ------------------------------------------------------------------ h-index
def test_hindex_examples():
    assert oracle.hindex([], 5) == 0
    assert oracle.hindex([3, 3, 3], 3) == 3
    assert oracle.hindex([1, 1, 1], 3) == 1
    assert oracle.hindex([5, 5], 5) == 2
    assert oracle.hindex([9, 9, 9, 9], 2) == 2          # capped
    assert oracle.hindex([0, 0, 0], 3) == 0
    assert oracle.hindex([4, 4, 1, 1], 4) == 2
    assert oracle.hindex([10, 8, 5, 4, 3], 5) == 4


def test_hindex_matches_sorted_definition():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        d = int(rng.integers(0, 40))
        vals = rng.integers(0, 50, d)
        cap = int(rng.integers(0, 60))
        assert oracle.hindex(vals, cap) == refimpl.hindex_sorted(vals, cap)


# ------------------------------------------------------------------ invariants at scale
def check_invariants(n, rp, col, core):
    deg = np.diff(rp)
    assert (core >= 0).all() and (core <= deg).all()
    rows = np.repeat(np.arange(n), deg)
    # {core >= k} induces minimum degree >= k
    for k in np.unique(core):
        inside = core >= k
        e = inside[rows] & inside[col]
        d_in = np.bincount(rows[e], minlength=n)
        assert (d_in[inside] >= k).all(), k
    # fixed point: core(v) is the h-index of its neighbours' corenesses
    np.testing.assert_array_equal(refimpl.hindex_uncapped_rows(n, rp, col, core), core)


@pytest.mark.parametrize("name", ["er10k"])
def test_workload_invariants_and_peeling(name):
    g = graphgen.workload(name)
    rp, col = oracle.csr_build(g.n, g.src, g.dst)
    core = oracle.coreness(g.n, rp, col)
    check_invariants(g.n, rp, col, core)
    np.testing.assert_array_equal(core, refimpl.coreness_peel_levels(g.n, rp, col))


def test_small_road_and_rmat_invariants_and_peeling():
    for g in (graphgen.damaged_grid(256, seed=3),
              graphgen.rmat(1 << 15, 16 << 15, 0.57, 0.19, 0.19, seed=2)):
        rp, col = oracle.csr_build(g.n, g.src, g.dst)
        core = oracle.coreness(g.n, rp, col)
        check_invariants(g.n, rp, col, core)
        np.testing.assert_array_equal(core, refimpl.coreness_peel_levels(g.n, rp, col))


def test_networkx_core_number():
    nx = pytest.importorskip("networkx")
    g = graphgen.workload("er10k")
    rp, col = oracle.csr_build(g.n, g.src, g.dst)
    core = oracle.coreness(g.n, rp, col)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(zip(g.src.tolist(), g.dst.tolist()))
    cn = nx.core_number(G)
    assert [cn[v] for v in range(g.n)] == core.tolist()


# ------------------------------------------------------------------ synchronous rounds
def test_sync_rounds_reach_coreness():
    rng = np.random.default_rng(5)
    for trial in range(30):
        n = int(rng.integers(1, 300))
        m = int(rng.integers(0, 5 * n + 1))
        src = rng.integers(0, n, m).astype(np.int32)
        dst = rng.integers(0, n, m).astype(np.int32)
        rp, col = oracle.csr_build(n, src, dst)
        core = oracle.coreness(n, rp, col)
        for refined in (False, True):
            r, est, _, _ = oracle.montresor_sync(n, rp, col, refined=refined)
            assert r >= 0
            np.testing.assert_array_equal(est, core)


def test_sync_round_step_semantics():
    """Each round: changed vertices take the capped h-index of the previous
    round's estimates; activation follows new_u < est[v]."""
    g = graphgen.rmat(1 << 11, 8 << 11, 0.57, 0.19, 0.19, seed=9)
    rp, col = oracle.csr_build(g.n, g.src, g.dst)
    n = g.n
    deg = np.diff(rp)
    total, _, fr, ch = oracle.montresor_sync(n, rp, col, record=1000)
    assert fr[0] == n
    prev = deg.astype(np.int32)
    for s in range(total):
        _, est, _, _ = oracle.montresor_sync(n, rp, col, max_rounds=s + 1)
        changed = np.nonzero(est != prev)[0]
        assert (est <= prev).all()
        assert changed.shape[0] == ch[s]
        for u in changed:
            nb = prev[col[rp[u]:rp[u + 1]]]
            assert est[u] == refimpl.hindex_sorted(nb, prev[u])
        # the next round's active set, from the activation rule
        act = set()
        for u in changed:
            for v in col[rp[u]:rp[u + 1]]:
                if est[u] < prev[v]:
                    act.add(int(v))
        if s + 1 < total:
            assert len(act) == fr[s + 1]
        else:
            assert len(act) == 0
        prev = est


def test_sync_round_step_semantics_refined():
    """Refined rule (Sec. IV, Further Optimizations, read as the conjunction
    new_u < est(v) <= old_u and decided after the round's updates, the extra
    barrier that passage mentions): every round's frontier is recomputed here
    from two consecutive rounds' estimates, independently of the oracle's
    bookkeeping, and must equal the oracle's next frontier.  The graphs hold
    many neighbours whose post-round estimate equals old_u exactly (the
    boundary of the <= ), and many whose pre-round value differs from the
    post-round one, so reading '<' for '<=', or the pre-round snapshot for the
    post-round value, changes a frontier size."""
    cases = [graphgen.rmat(1 << 11, 8 << 11, 0.57, 0.19, 0.19, seed=9),
             graphgen.union(graphgen.rmat(1 << 10, 6 << 10, 0.45, 0.22, 0.22, seed=21),
                            graphgen.planted(1 << 10, 60, 0.5, seed=22)),
             graphgen.damaged_grid(40, seed=23)]
    boundary_hits = 0
    stale_differs = 0
    for g in cases:
        rp, col = oracle.csr_build(g.n, g.src, g.dst)
        n = g.n
        deg = np.diff(rp)
        total, _, fr, ch = oracle.montresor_sync(n, rp, col, refined=True, record=1000)
        assert total >= 1 and fr[0] == n
        prev = deg.astype(np.int32)
        for s in range(total):
            _, est, _, _ = oracle.montresor_sync(n, rp, col, max_rounds=s + 1, refined=True)
            changed = np.nonzero(est != prev)[0]
            assert (est <= prev).all()
            assert changed.shape[0] == ch[s]
            act = set()
            for u in changed:
                nbrs = col[rp[u]:rp[u + 1]]
                # the round computes from the previous round's estimates
                assert est[u] == refimpl.hindex_sorted(prev[nbrs], prev[u])
                old_u, new_u = int(prev[u]), int(est[u])
                for v in nbrs:
                    x = int(est[v])          # v's value after this round
                    if new_u < x <= old_u:
                        act.add(int(v))
                    boundary_hits += int(x == old_u)
                    stale_differs += int((new_u < int(prev[v]) <= old_u) != (new_u < x <= old_u))
            if s + 1 < total:
                assert len(act) == fr[s + 1], (g.name, s)
            else:
                assert len(act) == 0
            prev = est
    # the cases exercise both readings that a slip would change
    assert boundary_hits > 100 and stale_differs > 10


def test_sync_start_from_degree_matters_on_cycle():
    n = 9
    rp, col = csr_of(n, cycle(n))
    r, est, fr, _ = oracle.montresor_sync(n, rp, col, record=10)
    assert (est == 2).all()
    assert r == 1 and fr.tolist() == [n]     # degrees are already the fixed point


def test_refined_activation_never_activates_more():
    g = graphgen.rmat(1 << 13, 16 << 13, 0.57, 0.19, 0.19, seed=4)
    rp, col = oracle.csr_build(g.n, g.src, g.dst)
    r1, e1, f1, _ = oracle.montresor_sync(g.n, rp, col, record=10000)
    r2, e2, f2, _ = oracle.montresor_sync(g.n, rp, col, refined=True, record=10000)
    np.testing.assert_array_equal(e1, e2)
    assert f2.sum() <= f1.sum()
