"""kcore_run_noalloc, the entry point for callers that cannot allocate device
memory, against kcore_run (GPU).

Callers that reserved the whole device for their own memory plan, or that run
where an allocation would stall or fail, call kcore_run_noalloc: its working
memory is a fixed array compiled into the library.  It must give exactly the
coreness kcore_run gives (tolerance zero: coreness is an integer and unique),
also when called twice in a row, since every call reuses the array the
previous call left behind.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import paper_2512_00233_gb300 as K
from paper_2512_00233_gb300 import _lib

pytestmark = pytest.mark.gpu


def clean_csr_and_reference(g0, rp_bytes):
    """The cleaned CSR and its coreness from the allocating entry points."""
    with K.Graph.from_coo(g0.n, g0.src, g0.dst, rp_bytes) as g:
        rp, col = g.csr()
        ref = g.run().cpu().numpy()
    return rp, col, ref


def run_noalloc(torch, n, rp, col):
    rp_d = torch.from_numpy(rp).cuda()
    col_d = torch.from_numpy(col).cuda()
    out = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    st = K.lib().kcore_run_noalloc(n, rp_d.data_ptr(), rp.dtype.itemsize, col_d.data_ptr(),
                                   out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st, out[:n].cpu().numpy()


def test_noalloc_matches_kcore_run_on_two_calls_in_a_row():
    import torch
    assert torch.cuda.is_available()
    big = graphgen.union(graphgen.rmat(1 << 18, 10 << 18, 0.57, 0.19, 0.19, seed=31),
                         graphgen.planted(1 << 18, 600, 0.5, seed=32))
    small = graphgen.damaged_grid(300, seed=33)
    for g0, rp_bytes in ((big, 8), (small, 4)):
        rp, col, ref = clean_csr_and_reference(g0, rp_bytes)
        assert g0.n <= _lib.KCORE_NOALLOC_MAX_N
        st, got = run_noalloc(torch, g0.n, rp, col)
        assert st == K.KCORE_OK, K.lib().kcore_last_error()
        np.testing.assert_array_equal(got, ref)


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    n = _lib.KCORE_NOALLOC_MAX_N + 1
    st = K.lib().kcore_run_noalloc(n, ctypes.c_void_p(16), 4, ctypes.c_void_p(16),
                                   ctypes.c_void_p(16), torch.cuda.current_stream().cuda_stream)
    assert st == K.KCORE_ERR_INVALID
    assert b"KCORE_NOALLOC_MAX_N" in K.lib().kcore_last_error()
