"""Batch / serving engine (continuous batching) on the GPU.

Every result must equal the oracle's coreness and the result the same graph
gets alone (tolerance zero: coreness is unique), whatever else shares the
arena and whenever the graph arrives.
"""
import time

import numpy as np
import pytest

import graphgen
import oracle
import paper_2512_00233_gb300 as K

pytestmark = pytest.mark.gpu


def stream(count, nmax, seed=0):
    return [graphgen.stream_graph(i, seed=seed, nmin=100, nmax=nmax) for i in range(count)]


def oracle_core(g):
    rp, col = oracle.csr_build(g.n, g.src, g.dst)
    return oracle.coreness(g.n, rp, col)


def alone(g):
    with K.Graph.from_coo(g.n, g.src, g.dst) as gg:
        return gg.run(device=False)


@pytest.mark.parametrize("staging", [0, 1 << 18, -1])
def test_batch_results_match_oracle_and_alone(staging):
    """staging: the default page-locked pool; one that holds only some of the
    graphs (the rest use pageable memory, mixed within one admission); none."""
    graphs = stream(40, 20000, seed=3)
    opts = K.default_serve_options(mem_budget=256 << 20, chunk_sweeps=4, host_staging=staging)
    with K.BatchEngine(opts) as eng:
        tickets = [eng.submit_coo(g.n, g.src, g.dst) for g in graphs]
        for g, t in zip(graphs, tickets):
            st, core = eng.poll(t, g.n, timeout_us=-1)
            assert st == K.KCORE_OK, K.lib().kcore_last_error()
            np.testing.assert_array_equal(core, oracle_core(g))
            np.testing.assert_array_equal(core, alone(g))
        s = eng.stats()
    assert s["completed"] == len(graphs) and s["failed"] == 0
    assert s["launches"] >= 1 and s["latency_p99_ms"] >= s["latency_p50_ms"] > 0


def test_serve_autotuner_returns_a_timed_candidate_with_oracle_results():
    """The batch engine's tuner (coordinate descent: sweeps per launch, the
    cleaner its admissions use) times every candidate once per pass and
    returns one of them; the engine under the result gives the oracle's
    coreness for every graph."""
    from paper_2512_00233_gb300 import autotune
    graphs = stream(24, 20000, seed=11)
    base = K.default_serve_options(mem_budget=256 << 20, chunk_sweeps=8)
    space = {"chunk_sweeps": [4, 16], "build_sort": [1, -1]}
    best, trials = autotune.autotune_serve(graphs, base, reps=1, space=space)
    assert (trials[0][0], trials[0][1]) == ("base", None) and len(trials) == 5
    assert all(rate > 0 for _, _, rate in trials)
    assert best.chunk_sweeps in (4, 8, 16) and best.sweep.build_sort in (0, 1, -1)
    with K.BatchEngine(best) as eng:
        tickets = [eng.submit_coo(g.n, g.src, g.dst) for g in graphs]
        for g, t in zip(graphs, tickets):
            st, core = eng.poll(t, g.n, timeout_us=-1)
            assert st == K.KCORE_OK, K.lib().kcore_last_error()
            np.testing.assert_array_equal(core, oracle_core(g))


def test_arrivals_while_others_run_are_admitted_and_unchanged():
    """Waves of submissions while earlier graphs are resident; one sweep per
    chunk forces admissions between the sweeps of graphs already running."""
    graphs = stream(30, 60000, seed=5)
    expect = [alone(g) for g in graphs]
    opts = K.default_serve_options(mem_budget=512 << 20, chunk_sweeps=1)
    with K.BatchEngine(opts) as eng:
        tickets = []
        for w in range(3):
            for g in graphs[w * 10:(w + 1) * 10]:
                tickets.append(eng.submit_coo(g.n, g.src, g.dst))
            time.sleep(0.002)
        for g, t, e in zip(graphs, tickets, expect):
            st, core = eng.poll(t, g.n, timeout_us=-1)
            assert st == K.KCORE_OK
            np.testing.assert_array_equal(core, e)
        s = eng.stats()
    assert s["completed"] == len(graphs)
    assert s["launches"] > 3


def test_caller_driven_engine_and_csr_submission():
    graphs = stream(12, 5000, seed=9)
    opts = K.default_serve_options(mem_budget=64 << 20, start_thread=0, chunk_sweeps=8)
    with K.BatchEngine(opts) as eng:
        tickets = []
        for g in graphs:
            rp, col = oracle.csr_build(g.n, g.src, g.dst)
            tickets.append(eng.submit_csr(g.n, rp, col))
        steps = 0
        while eng.step() > 0:
            steps += 1
            assert steps < 10000
        for g, t in zip(graphs, tickets):
            st, core = eng.poll(t, g.n, timeout_us=0)
            assert st == K.KCORE_OK
            np.testing.assert_array_equal(core, oracle_core(g))


def test_tight_arena_reuses_freed_space():
    """An arena that holds only a few graphs at a time must still finish all of
    them, reusing the ranges that finished graphs free."""
    graphs = stream(25, 30000, seed=11)
    opts = K.default_serve_options(mem_budget=24 << 20, chunk_sweeps=4)
    with K.BatchEngine(opts) as eng:
        tickets = [eng.submit_coo(g.n, g.src, g.dst) for g in graphs]
        for g, t in zip(graphs, tickets):
            st, core = eng.poll(t, g.n, timeout_us=-1)
            assert st == K.KCORE_OK
            np.testing.assert_array_equal(core, oracle_core(g))


def test_admission_errors_and_cancel():
    opts = K.default_serve_options(mem_budget=16 << 20, max_queue=2, start_thread=0)
    with K.BatchEngine(opts) as eng:
        big = graphgen.er(2_000_000, 100, seed=1)          # never fits 16 MiB
        with pytest.raises(K.KCoreError) as e:
            eng.submit_coo(big.n, big.src, big.dst)
        assert e.value.status == K.KCORE_ERR_AGAIN
        g = graphgen.er(1000, 4000, seed=2)
        t1 = eng.submit_coo(g.n, g.src, g.dst)
        t2 = eng.submit_coo(g.n, g.src, g.dst)
        with pytest.raises(K.KCoreError) as e:             # queue of 2 is full
            eng.submit_coo(g.n, g.src, g.dst)
        assert e.value.status == K.KCORE_ERR_AGAIN
        assert eng.cancel(t2) == K.KCORE_OK
        st, core = eng.poll(t1, g.n, timeout_us=-1)
        assert st == K.KCORE_OK
        np.testing.assert_array_equal(core, oracle_core(g))
        st, _ = eng.poll(t2, g.n, timeout_us=-1)
        assert st == K.KCORE_ERR_CANCELLED
        with pytest.raises(K.KCoreError):
            eng.submit_coo(5, np.array([0, 7], np.int32), np.array([1, 1], np.int32))


def stream_range_indices():
    """Indices of the 20,000-graph stream (n log-uniform in [100, 200000],
    ER / R-MAT / damaged grid) covering its whole range: the three largest and
    the two smallest graphs of each family, and the first 30 of the stream."""
    params = [graphgen.stream_params(i) for i in range(20000)]
    pick = list(range(30))
    for fam in graphgen.STREAM_FAMILIES:
        by_n = sorted((n, i) for i, (n, f) in enumerate(params) if f == fam)
        pick += [i for _, i in by_n[-3:]] + [i for _, i in by_n[:2]]
    return sorted(set(pick)), params


def test_stream_full_range_in_waves_matches_oracle_and_overlaps():
    """Graphs from the whole size range of the stream (up to n = 199,809, all
    three families) submitted in waves while earlier ones are resident, into
    an arena that holds several of the largest at once.  Every result must
    equal the oracle's coreness (the unique fixed point of the iteration,
    Alg. 1), and the engine must have placed graphs while others were still
    resident and unfinished: for some pair, B's first launch lies inside A's
    launches."""
    idx, params = stream_range_indices()
    assert max(params[i][0] for i in idx) > 199_000
    assert {params[i][1] for i in idx} == set(graphgen.STREAM_FAMILIES)
    graphs = [graphgen.stream_graph(i) for i in idx]
    opts = K.default_serve_options(mem_budget=96 << 20, chunk_sweeps=2)
    waves = [graphs[j::3] for j in range(3)]
    infos, results = [], []
    with K.BatchEngine(opts) as eng:
        tickets = []
        for w, wave in enumerate(waves):
            for g in wave:
                tickets.append((g, eng.submit_coo(g.n, g.src, g.dst)))
            if w + 1 < len(waves):          # the next wave arrives while this one runs
                t_end = time.perf_counter() + 5.0
                while eng.stats()["launches"] < 2 * (w + 1) and time.perf_counter() < t_end:
                    time.sleep(0.0005)
        for g, t in tickets:
            st, core, info = eng.poll_info(t, g.n, timeout_us=-1)
            assert st == K.KCORE_OK, K.lib().kcore_last_error()
            results.append((g, core))
            infos.append(info)
        s = eng.stats()
    for g, core in results:
        np.testing.assert_array_equal(core, oracle_core(g), err_msg=g.name)
    assert s["completed"] == len(graphs) and s["failed"] == 0
    assert s["admitted_while_busy"] > 0
    overlap = any(a["admit_launch"] < b["admit_launch"] < a["retire_launch"]
                  for a in infos for b in infos)
    assert overlap, "no graph was admitted while another was resident and unfinished"
    for info in infos:
        assert info["submit_s"] <= info["admit_s"] <= info["done_s"]
        assert 0 <= info["admit_launch"] < info["retire_launch"]


def test_freed_neighbour_range_reused_while_a_graph_is_resident():
    """Graphs admitted together sit next to each other in the arena.  Here a
    tiny graph H retires while its block neighbour G (a long path, which
    converges over many sweeps, with its middle vertex numbered last) is still
    resident, and a new graph X is placed into H's freed range.  G's last
    row must be unaffected: every result equals the oracle's coreness."""
    L = 4001
    order = list(range(L - 1))
    order.insert(L // 2, L - 1)                       # vertex L-1 in the middle of the path
    g_src = np.array(order[:-1], np.int32)
    g_dst = np.array(order[1:], np.int32)
    G = graphgen.EdgeList(L, g_src, g_dst, "path_middle_last")
    H = graphgen.EdgeList(3, np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32), "triangle")
    X = graphgen.EdgeList(2, np.array([0], np.int32), np.array([1], np.int32), "edge")
    opts = K.default_serve_options(mem_budget=32 << 20, start_thread=0, chunk_sweeps=1)
    with K.BatchEngine(opts) as eng:
        tg = eng.submit_coo(G.n, G.src, G.dst)
        th = eng.submit_coo(H.n, H.src, H.dst)          # same admission, right after G
        eng.step()
        steps = 1
        while eng.poll(th, H.n, timeout_us=0)[0] == K.KCORE_PENDING:
            eng.step()
            steps += 1
            assert steps < 100
        assert eng.stats()["resident"] == 1              # G is still running
        tx = eng.submit_coo(X.n, X.src, X.dst)           # fits into H's freed range
        while eng.step() > 0:
            steps += 1
            assert steps < 100000
        for g, t in ((G, tg), (X, tx)):
            st, core, info = eng.poll_info(t, g.n, timeout_us=0)
            assert st == K.KCORE_OK
            np.testing.assert_array_equal(core, oracle_core(g), err_msg=g.name)
        assert info["resident_at_admit"] == 1
