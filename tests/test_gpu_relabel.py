"""Vertex renumbering by degree (kcore_options.relabel) on the GPU.

Renumbering is internal to the library: coreness, the cleaned CSR and warm
starts all use the caller's ids.  Every result here must equal the oracle's
(Batagelj-Zaversnik coreness of the same graph, tolerance zero) whatever the
numbering the sweeps run in: descending and ascending degree order, the
automatic choice and the input's order, with the other knobs changed on a
renumbered graph.
"""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2512_00233_gb300 as K

pytestmark = pytest.mark.gpu


def heavy_graph():
    # 2m ~ 2.5 M entries, largest degree far above 32 x the average: the
    # automatic choice renumbers it
    return graphgen.union(graphgen.rmat(1 << 16, 20 << 16, 0.57, 0.19, 0.19, seed=61),
                          graphgen.planted(1 << 16, 400, 0.5, seed=62))


@pytest.fixture(scope="module")
def case():
    g0 = heavy_graph()
    rp, col = oracle.csr_build(g0.n, g0.src, g0.dst)
    core = oracle.coreness(g0.n, rp, col)
    deg = np.diff(rp)
    assert rp[-1] >= 1 << 20 and deg.max() >= 32 * deg.mean()
    return g0, rp, col, core


@pytest.mark.parametrize("relabel", [0, 1, 2, -1])
def test_every_order_gives_the_oracle_coreness(case, relabel):
    import torch
    g0, rp, col, core = case
    opts = K.default_options(relabel=relabel)
    with K.Graph.from_coo(g0.n, g0.src, g0.dst, 8, options=opts) as g:
        grp, gcol = g.csr()                       # the caller's ids
        np.testing.assert_array_equal(grp, rp)
        np.testing.assert_array_equal(gcol, col)
        np.testing.assert_array_equal(g.run().cpu().numpy(), core)
        np.testing.assert_array_equal(g.run(device=False), core)
        np.testing.assert_array_equal(g.run(refined=False).cpu().numpy(), core)
        for refined in (False, True):
            np.testing.assert_array_equal(g.run(sync_mode=True, refined=refined).cpu().numpy(), core)
        out = torch.empty(g0.n, dtype=torch.int32, device="cuda")
        for _ in range(2):                        # captured graph, replayed
            g.run(out=out, graph=True)
            np.testing.assert_array_equal(out.cpu().numpy(), core)
        st = g.stats()
        assert st["status"] == 0 and st["nnz"] == rp[-1]


def test_other_options_on_a_renumbered_graph(case):
    g0, rp, col, core = case
    with K.Graph.from_coo(g0.n, g0.src, g0.dst, 8, options=K.default_options(relabel=2)) as g:
        for opts in (dict(t_lo=4, t_hi=256), dict(block=256, med_chunk=16), dict(relabel=-1), {}):
            g.set_options(K.default_options(**opts))    # the numbering stays as made
            np.testing.assert_array_equal(g.run(device=False), core, err_msg=str(opts))
            np.testing.assert_array_equal(g.csr()[1], col)


def test_order_picker_and_small_graphs_keep_their_numbering(case):
    from paper_2512_00233_gb300 import autotune
    g0, rp, col, core = case
    best, times = autotune.pick_order(
        lambda r: K.Graph.from_coo(g0.n, g0.src, g0.dst, 8, options=K.default_options(relabel=r)), reps=1)
    assert best in (1, 2, -1) and set(times) == {1, 2, -1}
    # a graph below the automatic threshold, and one forced: same coreness
    small = graphgen.rmat(1 << 10, 8 << 10, 0.57, 0.19, 0.19, seed=63)
    srp, scol = oracle.csr_build(small.n, small.src, small.dst)
    score = oracle.coreness(small.n, srp, scol)
    for r in (0, 1, 2):
        with K.Graph.from_coo(small.n, small.src, small.dst, options=K.default_options(relabel=r)) as g:
            np.testing.assert_array_equal(g.run(device=False), score)
            np.testing.assert_array_equal(g.csr()[1], scol)


@pytest.mark.parametrize("relabel", [1, 2])
@pytest.mark.parametrize("device", [False, True])
def test_warm_starts_in_callers_ids(case, relabel, device):
    import torch
    g0, rp, col, core = case
    src = np.repeat(np.arange(g0.n, dtype=np.int32), np.diff(rp))
    keep = src < col
    a, b = src[keep], col[keep].astype(np.int32)
    rng = np.random.default_rng(relabel)
    drop = rng.random(a.shape[0]) < 0.01
    rp2, col2 = oracle.csr_build(g0.n, a[~drop], b[~drop])
    expect = oracle.coreness(g0.n, rp2, col2)
    ends = np.unique(np.concatenate([a[drop], b[drop]])).astype(np.int32)
    opts = K.default_options(relabel=relabel)
    with K.Graph.from_coo(g0.n, a[~drop], b[~drop], 8, options=opts) as g:
        start = core.astype(np.int32)
        if device:
            got = g.run_from(torch.from_numpy(start).cuda(), torch.from_numpy(ends).cuda()).cpu().numpy()
        else:
            got = g.run_from(start, ends, device=False)
        np.testing.assert_array_equal(got, expect)
        # insertions: old coreness + b with everything active (here b = 0 after
        # re-adding nothing: start = the new coreness itself is a fixed point)
        got = g.run_from(expect.astype(np.int32) + 1, None, device=False)
        np.testing.assert_array_equal(got, expect)


@pytest.mark.parametrize("opts", [dict(t_lo=2, t_hi=64, block=128), dict(tail_max=-1),
                                  dict(max_ctas=2, med_chunk=1), dict(t_lo=1, t_hi=1)])
def test_launch_shapes_with_renumbering(case, opts):
    g0, rp, col, core = case
    with K.Graph.from_coo(g0.n, g0.src, g0.dst, 8, options=K.default_options(relabel=1, **opts)) as g:
        np.testing.assert_array_equal(g.run().cpu().numpy(), core)
