"""GPU parity: the CUDA path (through the C ABI) against the oracle, bit-exact.

Coreness is an integer and unique (Def. 1), so the tolerance is zero
everywhere: every vertex must match the oracle's Batagelj-Zaversnik value and
the cleaned CSR must equal the oracle's host-built CSR entry for entry.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import oracle
import paper_2512_00233_gb300 as K
from tests import golden_io

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def gpu_coreness(n, src, dst, rp_bytes=4, options=None, device_out=True, sync_mode=False,
                 refined=False):
    with K.Graph.from_coo(n, np.asarray(src, np.int32), np.asarray(dst, np.int32), rp_bytes,
                          options) as g:
        out = g.run(device=device_out, sync_mode=sync_mode, refined=refined)
        res = out.cpu().numpy() if device_out else out
        return res, g.stats()


def oracle_of(n, src, dst):
    rp, col = oracle.csr_build(n, src, dst)
    return rp, col, oracle.coreness(n, rp, col)


# ------------------------------------------------------------------ fixtures, closed forms
@pytest.mark.parametrize("fx", golden_io.all_fixtures(), ids=lambda f: f["name"])
def test_golden_fixture(torch_cuda, fx):
    with K.Graph.from_coo(fx["n"], fx["src"], fx["dst"]) as g:
        assert g.run().cpu().tolist() == fx["coreness"]
        if "row_ptr" in fx:
            rp, col = g.csr()
            assert rp.tolist() == fx["row_ptr"] and col.tolist() == fx["col"]


def test_closed_forms(torch_cuda):
    def check(n, edges, expect):
        e = np.array(edges, np.int32).reshape(-1, 2)
        got, _ = gpu_coreness(n, e[:, 0], e[:, 1])
        assert (got == expect).all(), (n, expect)
    check(1, [], 0)
    check(7, [], 0)
    check(60, [(a, b) for a in range(60) for b in range(a + 1, 60)], 59)
    check(1000, [(i, (i + 1) % 1000) for i in range(1000)], 2)
    check(500, [(0, i) for i in range(1, 500)], 1)
    check(800, [(i, i + 1) for i in range(799)], 1)
    a, b = 7, 300
    check(a + b, [(i, a + j) for i in range(a) for j in range(b)], a)


def test_empty_graph(torch_cuda):
    with K.Graph.from_coo(0, np.zeros(0, np.int32), np.zeros(0, np.int32)) as g:
        assert g.n == 0 and g.nnz == 0
        out = g.run()
        assert out.numel() == 0


# ------------------------------------------------------------------ random graphs, all tiers
def random_graph(rng, n, m, hubs=0, hub_deg=0):
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    if hubs:
        hs = rng.integers(0, n, hubs * hub_deg).astype(np.int32)
        hd = np.repeat(rng.integers(0, n, hubs).astype(np.int32), hub_deg)
        src, dst = np.concatenate([src, hs]), np.concatenate([dst, hd])
    return src, dst


@pytest.mark.parametrize("seed", range(6))
def test_random_graphs_match_oracle(torch_cuda, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(50, 6000))
    m = int(rng.integers(n, 12 * n))
    src, dst = random_graph(rng, n, m, hubs=3, hub_deg=int(rng.integers(100, 3000)))
    rp, col, core = oracle_of(n, src, dst)
    with K.Graph.from_coo(n, src, dst) as g:
        grp, gcol = g.csr()
        np.testing.assert_array_equal(grp, rp)
        np.testing.assert_array_equal(gcol, col)
        np.testing.assert_array_equal(g.run().cpu().numpy(), core)
        np.testing.assert_array_equal(g.run(device=False), core)
        np.testing.assert_array_equal(g.run(refined=True).cpu().numpy(), core)


@pytest.mark.parametrize("refined", [False, True])
@pytest.mark.parametrize("opts", [
    dict(t_lo=1, t_hi=1),                  # everything above degree 1 in the CTA tier
    dict(t_lo=2, t_hi=32),
    dict(t_lo=8, t_hi=64, block=64),
    dict(t_lo=16, t_hi=256, block=256),
    dict(t_lo=16, t_hi=2048),              # staged warp tier up to degree 2048
    dict(t_lo=4, t_hi=1024, block=128),
    dict(tail_max=-1),                     # no single-CTA tail
    dict(tail_max=1 << 30),                # single CTA from the start
    dict(max_ctas=1),
    dict(max_ctas=3, low_chunk=1, med_chunk=1),
    dict(low_chunk=8, med_chunk=64),
])
def test_launch_shapes_and_tiers_match_oracle(torch_cuda, opts, refined):
    rng = np.random.default_rng(7)
    n = 20000
    src, dst = random_graph(rng, n, 6 * n, hubs=5, hub_deg=2000)
    g2 = graphgen.rmat(1 << 13, 8 << 13, 0.57, 0.19, 0.19, seed=3)
    src = np.concatenate([src, g2.src])
    dst = np.concatenate([dst, g2.dst])
    _, _, core = oracle_of(n, src, dst)
    got, st = gpu_coreness(n, src, dst, options=K.default_options(**opts), refined=refined)
    np.testing.assert_array_equal(got, core)
    assert st["status"] == 0 and st["sweeps"] >= 1


@pytest.mark.parametrize("refined", [False, True])
def test_hub_bracket_wider_than_histogram(torch_cuda, refined):
    """A dense block whose coreness exceeds 8192, and a hub X joined to the
    whole block and to 12,000 leaves.  In the first sweep X's estimate (its
    degree, 20,600) is more than twice its new value (about the block's
    coreness), so the value lies below pass 1's window and the power-of-two
    bracket [8192, 16383] is wider than the 4096-bucket histogram: the coarse
    buckets and the fine pass both run.  The block's own vertices land inside
    the window."""
    rng = np.random.default_rng(1)
    k = 8600
    a, b = np.triu_indices(k, 1)
    keep = rng.random(a.shape[0]) < 0.99
    x = k
    leaves = np.arange(k + 1, k + 1 + 12000)
    n = k + 1 + 12000 + 3000
    src = np.concatenate([a[keep], np.full(k, x), np.full(leaves.shape[0], x),
                          rng.integers(0, n, 20000)]).astype(np.int32)
    dst = np.concatenate([b[keep], np.arange(k), leaves,
                          rng.integers(0, n, 20000)]).astype(np.int32)
    _, _, core = oracle_of(n, src, dst)
    assert core.max() >= 8192 and 2 * core[x] < 20600
    got, _ = gpu_coreness(n, src, dst, refined=refined)
    np.testing.assert_array_equal(got, core)


def test_hub_early_exit_and_entries_read(torch_cuda):
    """Hubs whose estimate holds stop reading once they found k supporters:
    entries_read stays below the frontier degree sum, and the result is exact."""
    rng = np.random.default_rng(4)
    k = 600
    a, b = np.triu_indices(k, 1)
    n = 2_000_000
    hubs = np.arange(k, dtype=np.int32)
    # each clique member also gets many low-degree leaves after its clique edges
    leaf_src = np.repeat(hubs, 20000)
    leaf_dst = rng.integers(k, n, leaf_src.shape[0]).astype(np.int32)
    src = np.concatenate([a, leaf_src]).astype(np.int32)
    dst = np.concatenate([b, leaf_dst]).astype(np.int32)
    _, _, core = oracle_of(n, src, dst)
    got, st = gpu_coreness(n, src, dst)
    np.testing.assert_array_equal(got, core)
    assert st["entries_read"] < st["edges_scanned"]
    assert st["decrease"] > 0


def test_csr_input_paths(torch_cuda):
    rng = np.random.default_rng(3)
    n = 3000
    src, dst = random_graph(rng, n, 5 * n, hubs=2, hub_deg=700)
    rp, col, core = oracle_of(n, src, dst)
    # raw (directed, repeated, loops) CSR input: rows of the samples
    order = np.argsort(src, kind="stable")
    raw_rp = np.zeros(n + 1, np.int64)
    np.add.at(raw_rp, src.astype(np.int64) + 1, 1)
    raw_rp = np.cumsum(raw_rp)
    raw_col = dst[order]
    for rp_dtype in (np.int32, np.int64):
        with K.Graph.from_csr(n, raw_rp.astype(rp_dtype), raw_col) as g:
            assert g.row_ptr_bytes == np.dtype(rp_dtype).itemsize
            grp, gcol = g.csr()
            np.testing.assert_array_equal(grp, rp)
            np.testing.assert_array_equal(gcol, col)
            np.testing.assert_array_equal(g.run().cpu().numpy(), core)
    # already clean input, host and device
    with K.Graph.from_csr(n, rp, col, clean=True) as g:
        np.testing.assert_array_equal(g.run().cpu().numpy(), core)
    t = torch_cuda
    with K.Graph.from_csr(n, t.from_numpy(rp).cuda(), t.from_numpy(col).cuda(), clean=True) as g:
        np.testing.assert_array_equal(g.run().cpu().numpy(), core)
    with K.Graph.from_coo(n, t.from_numpy(src).cuda(), t.from_numpy(dst).cuda()) as g:
        np.testing.assert_array_equal(g.run().cpu().numpy(), core)


# ------------------------------------------------------------------ the two COO cleaners
SORTED, COUNTED = 1, -1   # build_sort: the sorted build / rows counted one by one


def cleaner_cases():
    rng = np.random.default_rng(77)
    cases = []
    # n a power of two (the largest id has every id bit set), hubs in every
    # row size class up to the hub radix path (> 16384 entries)
    src, dst = random_graph(rng, 1 << 12, 6 << 12, hubs=4, hub_deg=9000)
    src = np.concatenate([src, np.full(20000, 5, np.int32)])
    dst = np.concatenate([dst, rng.integers(0, 1 << 12, 20000).astype(np.int32)])
    cases.append(("pow2_hubs", 1 << 12, src, dst))
    # n just above a power of two, loops and repeats, isolated vertices at both ends
    n = (1 << 11) + 3
    a = rng.integers(100, n - 100, 4 * n).astype(np.int32)
    b = rng.integers(100, n - 100, 4 * n).astype(np.int32)
    a = np.concatenate([a, a[:500], np.arange(100, 400, dtype=np.int32)])
    b = np.concatenate([b, b[:500], np.arange(100, 400, dtype=np.int32)])
    cases.append(("loops_repeats", n, a, b))
    cases.append(("one_edge", 2, np.array([1, 1, 0], np.int32), np.array([0, 1, 1], np.int32)))
    cases.append(("only_loops", 4, np.arange(4, dtype=np.int32), np.arange(4, dtype=np.int32)))
    cases.append(("single_vertex", 1, np.zeros(3, np.int32), np.zeros(3, np.int32)))
    g = graphgen.rmat(1 << 13, 16 << 13, 0.57, 0.19, 0.19, seed=4)
    cases.append(("rmat13", g.n, g.src, g.dst))
    # vertices but no samples at all
    cases.append(("no_samples", 5, np.zeros(0, np.int32), np.zeros(0, np.int32)))
    # 200,000 samples of 500 edges: the distinct edges fill one tile of the
    # sorted keys and the dropped repeats span dozens
    e = rng.integers(0, 300, (500, 2)).astype(np.int32)
    pick = rng.integers(0, 500, 200000)
    cases.append(("heavy_repeats", 300, e[pick, 0].copy(), e[pick, 1].copy()))
    return cases


@pytest.mark.parametrize("case", cleaner_cases(), ids=lambda c: c[0])
@pytest.mark.parametrize("rp_bytes", [4, 8])
def test_coo_cleaners_match_oracle(torch_cuda, case, rp_bytes):
    """Both COO cleaners (one radix sort of all entries; per-row counting and
    sorting) give the oracle's CSR entry for entry, and the same coreness."""
    _, n, src, dst = case
    rp, col, core = oracle_of(n, src, dst)
    for mode in (SORTED, COUNTED, 0):
        opts = K.default_options(build_sort=mode) if mode else None
        with K.Graph.from_coo(n, src, dst, rp_bytes, options=opts) as g:
            grp, gcol = g.csr()
            np.testing.assert_array_equal(grp, rp, err_msg=str(mode))
            np.testing.assert_array_equal(gcol, col, err_msg=str(mode))
            np.testing.assert_array_equal(g.run().cpu().numpy(), core, err_msg=str(mode))
    t = torch_cuda   # device samples through the sorted build
    with K.Graph.from_coo(n, t.from_numpy(np.asarray(src)).cuda(), t.from_numpy(np.asarray(dst)).cuda(),
                          rp_bytes, options=K.default_options(build_sort=SORTED)) as g:
        grp, gcol = g.csr()
        np.testing.assert_array_equal(grp, rp)
        np.testing.assert_array_equal(gcol, col)


@pytest.mark.parametrize("mode", [SORTED, COUNTED])
def test_coo_cleaners_reject_bad_ids(torch_cuda, mode):
    opts = K.default_options(build_sort=mode)
    for s, d in (([0, 5, 1], [1, 1, 2]), ([0, -1, 1], [1, 1, 2])):
        with pytest.raises(K.KCoreError) as e:
            K.Graph.from_coo(5, np.array(s, np.int32), np.array(d, np.int32), options=opts)
        assert e.value.status == K.KCORE_ERR_INVALID


def test_invalid_inputs_are_rejected(torch_cuda):
    with pytest.raises(K.KCoreError) as e:
        K.Graph.from_coo(5, np.array([0, 5], np.int32), np.array([1, 1], np.int32))
    assert e.value.status == K.KCORE_ERR_INVALID
    with pytest.raises(K.KCoreError):
        K.Graph.from_csr(3, np.array([0, 2, 1, 3], np.int32), np.array([1, 2, 0], np.int32))
    with pytest.raises(K.KCoreError):   # unsorted row with IN_CLEAN
        K.Graph.from_csr(3, np.array([0, 2, 3, 4], np.int32), np.array([2, 1, 0, 0], np.int32),
                         clean=True)
    with pytest.raises(K.KCoreError):
        K.default_options()  # valid
        K.Graph.from_coo(3, np.array([0], np.int32), np.array([1], np.int32),
                         options=K.default_options(t_lo=64))
    with pytest.raises(K.KCoreError):
        K.Graph.from_coo(3, np.array([0], np.int32), np.array([1], np.int32),
                         options=K.default_options(t_hi=4096))
    with pytest.raises(K.KCoreError):
        K.Graph.from_coo(3, np.array([0], np.int32), np.array([1], np.int32),
                         options=K.default_options(build_sort=2))


def test_repeated_runs_identical(torch_cuda):
    g0 = graphgen.rmat(1 << 14, 16 << 14, 0.57, 0.19, 0.19, seed=12)
    _, _, core = oracle_of(g0.n, g0.src, g0.dst)
    with K.Graph.from_coo(g0.n, g0.src, g0.dst) as g:
        for _ in range(5):
            np.testing.assert_array_equal(g.run().cpu().numpy(), core)


# ------------------------------------------------------------------ synchronous rounds
@pytest.mark.parametrize("refined", [False, True])
def test_sync_mode_matches_oracle_round_by_round(torch_cuda, refined):
    g0 = graphgen.rmat(1 << 12, 12 << 12, 0.57, 0.19, 0.19, seed=21)
    rp, col, core = oracle_of(g0.n, g0.src, g0.dst)
    rounds, est, fr, ch = oracle.montresor_sync(g0.n, rp, col, refined=refined, record=100000)
    assert rounds > 3
    with K.Graph.from_coo(g0.n, g0.src, g0.dst) as g:
        np.testing.assert_array_equal(g.run(sync_mode=True, refined=refined).cpu().numpy(), core)
        f, d, u = g.trace()
        assert g.stats()["sweeps"] == rounds
        np.testing.assert_array_equal(f, fr)
        np.testing.assert_array_equal(u, ch)
        for s in sorted({1, 2, 3, rounds // 2, rounds - 1}):
            _, est_s, _, _ = oracle.montresor_sync(g0.n, rp, col, max_rounds=s, refined=refined)
            g.set_options(K.default_options(max_sweeps=s))
            out = g.run(sync_mode=True, refined=refined, check_status=False)
            assert g.last_status == K.KCORE_ERR_NOT_CONVERGED
            np.testing.assert_array_equal(out.cpu().numpy(), est_s)


def test_sweep_cap_reports_not_converged(torch_cuda):
    g0 = graphgen.damaged_grid(64, seed=2)
    with K.Graph.from_coo(g0.n, g0.src, g0.dst, options=K.default_options(max_sweeps=1)) as g:
        out = g.run(check_status=False)
        assert g.last_status == K.KCORE_ERR_NOT_CONVERGED
        deg = np.diff(g.csr()[0])
        assert (out.cpu().numpy() <= deg).all()


def test_bounded_wait_reports_timeout_and_context_survives(torch_cuda):
    """A wait budget of 1 ns makes the grid barrier give up: the kernel must
    return KCORE_ERR_TIMEOUT (no hang, no fault) and the next run must work."""
    g0 = graphgen.rmat(1 << 15, 16 << 15, 0.57, 0.19, 0.19, seed=5)
    _, _, core = oracle_of(g0.n, g0.src, g0.dst)
    opts = K.default_options(timeout_s=1e-9, tail_max=-1)
    with K.Graph.from_coo(g0.n, g0.src, g0.dst, options=opts) as g:
        g.run(check_status=False)
        assert g.last_status == K.KCORE_ERR_TIMEOUT
        g.set_options(K.default_options())
        np.testing.assert_array_equal(g.run().cpu().numpy(), core)


# ------------------------------------------------------------------ named workloads
@pytest.mark.parametrize("name", ["er10k", "road2048", "rmat22", "rmat24_planted"])
def test_workload_full_size_matches_oracle(torch_cuda, name):
    g0 = graphgen.workload(name)
    rp, col, core = oracle_of(g0.n, g0.src, g0.dst)
    with K.Graph.from_coo(g0.n, g0.src, g0.dst, g0.meta["row_ptr_bytes"]) as g:
        grp, gcol = g.csr()
        np.testing.assert_array_equal(grp, rp)
        np.testing.assert_array_equal(gcol, col)
        np.testing.assert_array_equal(g.run().cpu().numpy(), core)
        st = g.stats()
        assert st["status"] == 0
        assert st["evaluated"] >= g0.n
        deg = np.diff(grp.astype(np.int64))
        assert st["decrease"] == int(deg.sum()) - int(core.astype(np.int64).sum())
        np.testing.assert_array_equal(g.run(refined=True).cpu().numpy(), core)
        assert g.stats()["decrease"] == st["decrease"]
