"""Dynamic core maintenance through warm starts (kcore_run_from).

After edge deletions the old coreness is an upper bound of the new one and
only the endpoints' neighbourhoods changed; after b insertions old core + b is
an upper bound.  Either way the iteration must end at the new graph's
coreness exactly (the oracle's), and a deletion restart must evaluate far
fewer vertices than a cold run.
"""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2512_00233_gb300 as K

pytestmark = pytest.mark.gpu


def undirected(g0):
    rp, col = oracle.csr_build(g0.n, g0.src, g0.dst)
    src = np.repeat(np.arange(g0.n, dtype=np.int32), np.diff(rp))
    keep = src < col
    return rp, col, src[keep], col[keep].astype(np.int32)


@pytest.mark.parametrize("device", [False, True])
@pytest.mark.parametrize("name_seed", [("rmat", 3), ("grid", 5)])
def test_deletions_restart_from_old_coreness(device, name_seed):
    import torch
    name, seed = name_seed
    g0 = graphgen.rmat(1 << 14, 12 << 14, 0.57, 0.19, 0.19, seed=seed) if name == "rmat" \
        else graphgen.damaged_grid(256, seed=seed)
    rp, col, a, b = undirected(g0)
    old = oracle.coreness(g0.n, rp, col)
    rng = np.random.default_rng(seed)
    drop = rng.random(a.shape[0]) < 0.01
    a2, b2 = a[~drop], b[~drop]
    rp2, col2 = oracle.csr_build(g0.n, a2, b2)
    expect = oracle.coreness(g0.n, rp2, col2)
    ends = np.unique(np.concatenate([a[drop], b[drop]])).astype(np.int32)
    with K.Graph.from_coo(g0.n, a2, b2) as g:
        cold = g.run(device=False)
        np.testing.assert_array_equal(cold, expect)
        cold_eval = g.stats()["evaluated"]
        if device:
            out = g.run_from(torch.from_numpy(old.astype(np.int32)).cuda(), torch.from_numpy(ends).cuda())
            got = out.cpu().numpy()
        else:
            got = g.run_from(old.astype(np.int32), ends, device=False)
        np.testing.assert_array_equal(got, expect)
        st = g.stats()
        assert st["status"] == 0 and st["evaluated"] < cold_eval // 2
        # a repeated cold run after the warm one is unaffected
        np.testing.assert_array_equal(g.run(device=False), expect)


def test_insertions_restart_from_old_coreness_plus_b():
    g0 = graphgen.rmat(1 << 13, 10 << 13, 0.57, 0.19, 0.19, seed=17)
    rp, col, a, b = undirected(g0)
    old = oracle.coreness(g0.n, rp, col)
    rng = np.random.default_rng(2)
    nb = 40
    ia = rng.integers(0, g0.n, nb).astype(np.int32)
    ib = rng.integers(0, g0.n, nb).astype(np.int32)
    a2, b2 = np.concatenate([a, ia]), np.concatenate([b, ib])
    rp2, col2 = oracle.csr_build(g0.n, a2, b2)
    expect = oracle.coreness(g0.n, rp2, col2)
    assert (expect >= old).all() and (expect > old).any()
    with K.Graph.from_coo(g0.n, a2, b2) as g:
        got = g.run_from((old + nb).astype(np.int32), None, device=False)
        np.testing.assert_array_equal(got, expect)
        got = g.run_from((old + nb).astype(np.int32), None, device=False, sync_mode=True)
        np.testing.assert_array_equal(got, expect)


def test_warm_start_cap_activates_neighbours():
    """A 4-cycle loses one edge: starting from the old coreness (2) with only
    the endpoints active, the endpoints' starts exceed their new degree; the
    library must treat that as a change so that the far vertices drop too."""
    src = np.array([0, 2, 3, 1], np.int32)
    dst = np.array([2, 3, 1, 0], np.int32)       # cycle 0-2-3-1-0
    keep = np.array([True, False, True, True])   # drop 2-3
    with K.Graph.from_coo(4, src[keep], dst[keep]) as g:
        got = g.run_from(np.full(4, 2, np.int32), np.array([2, 3], np.int32), device=False)
    np.testing.assert_array_equal(got, [1, 1, 1, 1])


def test_warm_start_rejects_bad_ids_and_graph_flag():
    g0 = graphgen.er(1000, 4000, seed=1)
    with K.Graph.from_coo(g0.n, g0.src, g0.dst) as g:
        core = g.run(device=False)
        g.run_from(core, np.array([5, 2000], np.int32), device=False, check_status=False)
        assert g.last_status == K.KCORE_ERR_INVALID
        np.testing.assert_array_equal(g.run(device=False), core)
        st = K.lib().kcore_run_from(g._h, core.ctypes.data, None, 0, core.ctypes.data,
                                    K.KCORE_GRAPH, None)
        assert st == K.KCORE_ERR_INVALID                 # graph capture is refused
