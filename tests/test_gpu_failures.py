"""Failure handling on the host (GPU tests; nothing here faults a GPU).

Allocation failures are injected with the test hook of include/kcore_test.h:
the k-th allocation request of the library fails as out-of-memory.  For
every request a call makes, the call must return KCORE_ERR_OOM, leave no
handle behind and give back to the library's device pool everything it took;
the next call must work.  A failed batch admission must fail only the graphs
of that admission and leave the resident ones running.  kcore_poll with a
finite timeout reports KCORE_PENDING while the work is resident.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import oracle
import paper_2512_00233_gb300 as K

pytestmark = pytest.mark.gpu


def pool_used():
    u, r = ctypes.c_int64(), ctypes.c_int64()
    assert K.lib().kcore_test_pool_usage(ctypes.byref(u), ctypes.byref(r)) == K.KCORE_OK
    return u.value


def requests_of(call):
    """Allocation requests one successful call makes (its result is released)."""
    L = K.lib()
    L.kcore_test_fail_alloc(0)
    obj = call()
    n = L.kcore_test_alloc_count()
    if obj is not None:
        obj.close()
    return n


def fail_each_request(call, what):
    """Fails every allocation request of `call` in turn."""
    L = K.lib()
    total = requests_of(call)
    assert total >= 1, what
    base = pool_used()
    for k in range(1, total + 1):
        L.kcore_test_fail_alloc(k)
        with pytest.raises(K.KCoreError) as e:
            obj = call()
            obj.close()
        L.kcore_test_fail_alloc(0)
        assert e.value.status == K.KCORE_ERR_OOM, (what, k, str(e.value))
        assert pool_used() == base, (what, k, "pool usage not restored")
    return total


def oracle_core(g):
    rp, col = oracle.csr_build(g.n, g.src, g.dst)
    return oracle.coreness(g.n, rp, col)


def test_create_and_run_report_oom_and_roll_back():
    import torch
    torch.cuda.set_device(0)
    cases = [graphgen.rmat(1 << 14, 16 << 14, 0.57, 0.19, 0.19, seed=41),   # sorted cleaner
             graphgen.damaged_grid(200, seed=42)]                           # counted cleaner
    for g0 in cases:
        expect = oracle_core(g0)
        rp, col = oracle.csr_build(g0.n, g0.src, g0.dst)
        src_d, dst_d = torch.from_numpy(g0.src).cuda(), torch.from_numpy(g0.dst).cuda()
        calls = {
            "create_coo host": lambda: K.Graph.from_coo(g0.n, g0.src, g0.dst, 8),
            "create_coo device": lambda: K.Graph.from_coo(g0.n, src_d, dst_d, 4),
            "create raw csr": lambda: K.Graph.from_csr(g0.n, rp, col),
            "create clean csr": lambda: K.Graph.from_csr(g0.n, rp.astype(np.int32), col, clean=True),
        }
        for what, call in calls.items():
            fail_each_request(call, what)
            with call() as g:                       # and then it works
                np.testing.assert_array_equal(g.run(device=False), expect)
        # runs that allocate: the first synchronous run (update lists) and a
        # warm start from host arrays (uploads)
        with K.Graph.from_coo(g0.n, g0.src, g0.dst) as g:
            L = K.lib()
            out = np.empty(g0.n, np.int32)
            for k in (1, 2):                        # the two update lists, in turn
                L.kcore_test_fail_alloc(k)
                with pytest.raises(K.KCoreError) as e:
                    g.run(out=out, sync_mode=True)
                L.kcore_test_fail_alloc(0)
                assert e.value.status == K.KCORE_ERR_OOM
            np.testing.assert_array_equal(g.run(out=out, sync_mode=True), expect)
            start = (expect + 1).astype(np.int32)
            L.kcore_test_fail_alloc(1)
            with pytest.raises(K.KCoreError) as e:
                g.run_from(start, out=out)
            L.kcore_test_fail_alloc(0)
            assert e.value.status == K.KCORE_ERR_OOM
            np.testing.assert_array_equal(g.run_from(start, out=out), expect)
    K.lib().kcore_test_fail_alloc(0)


def test_batch_create_oom_and_failed_admission_rolls_back():
    L = K.lib()
    opts = K.default_serve_options(mem_budget=64 << 20, start_thread=0, chunk_sweeps=1)
    # every device allocation of the engine itself
    n_req = requests_of(lambda: K.BatchEngine(opts))
    base = pool_used()
    for k in range(1, n_req + 1):
        L.kcore_test_fail_alloc(k)
        try:
            eng = K.BatchEngine(opts)
        except K.KCoreError as e:
            assert e.status == K.KCORE_ERR_OOM
        else:   # the failed request was the staging pool: pageable memory instead
            eng.close()
        L.kcore_test_fail_alloc(0)
        assert pool_used() == base
    a = graphgen.rmat(1 << 13, 8 << 13, 0.57, 0.19, 0.19, seed=43)
    b = graphgen.er(5000, 20000, seed=44)
    c = graphgen.damaged_grid(90, seed=45)
    with K.BatchEngine(opts) as eng:
        ta = eng.submit_coo(a.n, a.src, a.dst)
        eng.step()                                   # a is resident, not finished
        s0 = eng.stats()
        assert s0["resident"] == 1
        tb = eng.submit_coo(b.n, b.src, b.dst)
        L.kcore_test_fail_alloc(1)                   # b's admission cannot allocate
        eng.step()
        L.kcore_test_fail_alloc(0)
        st, core, info = eng.poll_info(tb, b.n, timeout_us=0)
        assert st == K.KCORE_ERR_OOM
        s1 = eng.stats()
        assert s1["failed"] == 1 and s1["resident"] <= 1
        tc = eng.submit_coo(c.n, c.src, c.dst)       # later admissions work
        while eng.step() > 0:
            pass
        st, core = eng.poll(ta, a.n, timeout_us=0)
        assert st == K.KCORE_OK
        np.testing.assert_array_equal(core, oracle_core(a))
        st, core = eng.poll(tc, c.n, timeout_us=0)
        assert st == K.KCORE_OK
        np.testing.assert_array_equal(core, oracle_core(c))
        s2 = eng.stats()
        assert s2["resident"] == 0 and s2["completed"] == 2


def test_poll_with_a_finite_timeout_reports_pending():
    """A caller-driven engine with a resident graph: poll(timeout 0) is
    PENDING; a poll with a finite timeout drives the engine until then and is
    PENDING or OK; with the engine thread, a 1 us poll on a large graph is
    PENDING, and a blocking poll then returns the oracle's coreness."""
    g = graphgen.rmat(1 << 17, 16 << 17, 0.57, 0.19, 0.19, seed=46)
    expect = oracle_core(g)
    opts = K.default_serve_options(mem_budget=256 << 20, start_thread=0, chunk_sweeps=1)
    with K.BatchEngine(opts) as eng:
        t = eng.submit_coo(g.n, g.src, g.dst)
        assert eng.poll(t, g.n, timeout_us=0)[0] == K.KCORE_PENDING
        eng.step()
        assert eng.poll(t, g.n, timeout_us=0)[0] == K.KCORE_PENDING
        st, core = eng.poll(t, g.n, timeout_us=200)
        assert st in (K.KCORE_PENDING, K.KCORE_OK)
        if st == K.KCORE_PENDING:
            st, core = eng.poll(t, g.n, timeout_us=-1)
        assert st == K.KCORE_OK
        np.testing.assert_array_equal(core, expect)
    opts = K.default_serve_options(mem_budget=256 << 20, chunk_sweeps=1)
    with K.BatchEngine(opts) as eng:
        t = eng.submit_coo(g.n, g.src, g.dst)
        assert eng.poll(t, g.n, timeout_us=1)[0] == K.KCORE_PENDING
        st, core = eng.poll(t, g.n, timeout_us=-1)
        assert st == K.KCORE_OK
        np.testing.assert_array_equal(core, expect)
