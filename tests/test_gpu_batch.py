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
