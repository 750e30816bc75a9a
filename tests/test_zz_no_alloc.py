"""kcore_run_noalloc, the entry point for callers that cannot allocate device
memory (GPU).

Who needs it: a serving process that reserved the whole device for its own
memory plan up front, a real-time loop that must not stall on the
allocator, code running inside another allocator's callback.  Such callers
call kcore_run_noalloc, whose working memory is a fixed array compiled into
the library.  Checked here, through the C ABI:
  - its coreness equals the oracle's (Batagelj-Zaversnik) exactly, on two
    calls in a row (every call reuses what the previous call left in the
    array) and equals kcore_run's; tolerance zero, since the coreness is an
    integer and unique;
  - after the preparation call (n = 0), calls change neither the device's
    free memory nor torch's reserved memory: nothing is allocated;
  - a CSR that is not clean (a self-loop, an unsorted row, an id out of
    range) is refused with KCORE_ERR_INVALID by the device-side checks;
  - sizes beyond the array are refused before any device work.
This file runs last (its name sorts last), alone or after the other tests.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import oracle
import paper_2512_00233_gb300 as K
from paper_2512_00233_gb300 import _lib

pytestmark = pytest.mark.gpu


def oracle_csr_and_coreness(g0):
    rp, col = oracle.csr_build(g0.n, g0.src, g0.dst)
    return rp, col, oracle.coreness(g0.n, rp, col)


def call(torch, n, rp_d, rp_bytes, col_d, out):
    return K.lib().kcore_run_noalloc(n, rp_d.data_ptr(), rp_bytes, col_d.data_ptr(),
                                     out.data_ptr(), torch.cuda.current_stream().cuda_stream)


def prepare(torch):
    st = K.lib().kcore_run_noalloc(0, None, 4, None, None, torch.cuda.current_stream().cuda_stream)
    assert st == K.KCORE_OK, K.lib().kcore_last_error()


def test_noalloc_matches_oracle_on_two_calls_in_a_row_and_allocates_nothing():
    import torch
    assert torch.cuda.is_available()
    prepare(torch)
    big = graphgen.union(graphgen.rmat(1 << 18, 10 << 18, 0.57, 0.19, 0.19, seed=31),
                         graphgen.planted(1 << 18, 600, 0.5, seed=32))
    small = graphgen.damaged_grid(300, seed=33)
    for g0, rp_bytes in ((big, 8), (small, 4)):
        rp, col, expect = oracle_csr_and_coreness(g0)
        assert g0.n <= _lib.KCORE_NOALLOC_MAX_N
        rp_d = torch.from_numpy(rp.astype(np.int64 if rp_bytes == 8 else np.int32)).cuda()
        col_d = torch.from_numpy(col).cuda()
        outs = [torch.full((g0.n,), -1, dtype=torch.int32, device="cuda") for _ in range(2)]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        reserved0 = torch.cuda.memory_reserved()
        for out in outs:
            st = call(torch, g0.n, rp_d, rp_bytes, col_d, out)
            assert st == K.KCORE_OK, K.lib().kcore_last_error()
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0, "kcore_run_noalloc changed free device memory"
            assert torch.cuda.memory_reserved() == reserved0
        for out in outs:
            np.testing.assert_array_equal(out.cpu().numpy(), expect)
        # and the allocating entry point gives the same
        with K.Graph.from_csr(g0.n, rp.astype(np.int64 if rp_bytes == 8 else np.int32), col,
                              clean=True) as g:
            np.testing.assert_array_equal(g.run().cpu().numpy(), expect)


def test_noalloc_refuses_a_csr_that_is_not_clean():
    import torch
    prepare(torch)
    g0 = graphgen.rmat(1 << 12, 8 << 12, 0.57, 0.19, 0.19, seed=34)
    rp, col, expect = oracle_csr_and_coreness(g0)
    deg = np.diff(rp)
    u = int(np.argmax(deg))            # a row with several entries
    b = int(rp[u])
    assert deg[u] >= 3
    loop = col.copy()
    loop[b + 1] = u                     # a self-loop (the row may then be unsorted too)
    unsorted = col.copy()
    unsorted[b], unsorted[b + 1] = col[b + 1], col[b]
    out_of_range = col.copy()
    out_of_range[-1] = g0.n
    rp_d = torch.from_numpy(rp).cuda()
    out = torch.empty(g0.n, dtype=torch.int32, device="cuda")
    for bad in (loop, unsorted, out_of_range):
        st = call(torch, g0.n, rp_d, 8, torch.from_numpy(bad).cuda(), out)
        assert st == K.KCORE_ERR_INVALID
        assert b"not clean" in K.lib().kcore_last_error()
    # the array is fine afterwards: a clean call gives the coreness
    st = call(torch, g0.n, rp_d, 8, torch.from_numpy(col).cuda(), out)
    assert st == K.KCORE_OK, K.lib().kcore_last_error()
    np.testing.assert_array_equal(out.cpu().numpy(), expect)


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    n = _lib.KCORE_NOALLOC_MAX_N + 1
    st = K.lib().kcore_run_noalloc(n, ctypes.c_void_p(16), 4, ctypes.c_void_p(16),
                                   ctypes.c_void_p(16), torch.cuda.current_stream().cuda_stream)
    assert st == K.KCORE_ERR_INVALID
    assert b"KCORE_NOALLOC_MAX_N" in K.lib().kcore_last_error()
