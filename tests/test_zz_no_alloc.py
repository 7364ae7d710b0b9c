"""The allocation-free Gram entry point, tps_gram_noalloc, against tps_gram.

tps_gram_noalloc exists for callers that cannot allocate device memory (their device
memory belongs to a memory manager that hands all of it out up front).  It keeps its
partial sums in a fixed array inside the library, so this test checks that two calls in
a row -- the second one reusing the array the first one left behind -- both agree with
the context-based tps_gram, and that sizes beyond its limits are refused.  The file is
named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import torch, require_gpu, dev, host
from paper_2111_02534_gb300.inputs import random_block

pytestmark = pytest.mark.gpu


def _gram_with_context(ctx, A, p, B, q, nrows):
    G = torch.full((q, p), np.nan, dtype=torch.float64, device="cuda")
    ctx.gram(dev(A), p, dev(B), q, nrows, G)
    return host(G)


def test_noalloc_gram_matches_context_gram_twice():
    require_gpu()
    from paper_2111_02534_gb300 import tps
    ctx = tps.Context(1, 0)
    cases = [(131584, 24, 8, 1), (1000003, 64, 5, 2)]   # second call reuses the scratch array
    for nrows, p, q, seed in cases:
        A = random_block(p, nrows, seed)
        B = random_block(q, nrows, seed + 10)
        ref = _gram_with_context(ctx, A, p, B, q, nrows)
        G = torch.full((q, p), np.nan, dtype=torch.float64, device="cuda")
        # keep the device copies referenced until the kernel has read them (a temporary
        # would return its memory to torch's cache, where the next copy could reuse it)
        Ad, Bd = dev(A), dev(B)
        st = tps._lib.tps_gram_noalloc(ctypes.c_void_p(Ad.data_ptr()), nrows, p,
                                       ctypes.c_void_p(Bd.data_ptr()), nrows, q, nrows,
                                       ctypes.c_void_p(G.data_ptr()), p,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == tps.OK
        got = host(G)
        del Ad, Bd
        scale = max(1.0, np.sqrt(nrows)) * max(1.0, np.abs(ref).max())
        assert np.max(np.abs(got - ref)) <= 1e-14 * scale
        assert np.max(np.abs(got.T - A @ B.T)) <= 1e-14 * scale
    ctx.close()


def _noalloc(tps, Ad, lda, p, Bd, ldb, q, nrows, G, ldg):
    return tps._lib.tps_gram_noalloc(ctypes.c_void_p(Ad.data_ptr()), lda, p,
                                     ctypes.c_void_p(Bd.data_ptr()), ldb, q, nrows,
                                     ctypes.c_void_p(G.data_ptr()), ldg,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_gram_strided_and_empty():
    """Leading dimensions larger than the row count (A, B) and than p (G): only the p x q
    block of G is written and G's padding rows keep their values; with no rows G is zero."""
    require_gpu()
    from paper_2111_02534_gb300 import tps
    nrows, p, q, lda, ldb, ldg = 20011, 7, 5, 20016, 20023, 11
    A = random_block(p, lda, 31)
    B = random_block(q, ldb, 32)
    Ad, Bd = dev(A), dev(B)
    G = torch.full((q, ldg), -7.0, dtype=torch.float64, device="cuda")   # column-major, ld 11
    assert _noalloc(tps, Ad, lda, p, Bd, ldb, q, nrows, G, ldg) == tps.OK
    got = host(G)
    ref = A[:, :nrows] @ B[:, :nrows].T
    assert np.max(np.abs(got[:, :p].T - ref)) <= 1e-14 * np.sqrt(nrows) * max(1.0, np.abs(ref).max())
    assert np.all(got[:, p:] == -7.0)
    G0 = torch.full((q, ldg), np.nan, dtype=torch.float64, device="cuda")
    assert _noalloc(tps, Ad, lda, p, Bd, ldb, q, 0, G0, ldg) == tps.OK
    g0 = host(G0)
    assert np.all(g0[:, :p] == 0.0) and np.all(np.isnan(g0[:, p:]))
    del Ad, Bd


def test_noalloc_gram_refuses_sizes_beyond_its_limit():
    require_gpu()
    from paper_2111_02534_gb300 import tps
    A = torch.zeros(65, 8, dtype=torch.float64, device="cuda")
    G = torch.zeros(65 * 65, dtype=torch.float64, device="cuda")
    with pytest.raises(tps.TpsError) as e:
        tps.gram_noalloc(A, 65, A, 1, 8, G, ldg=65)
    assert e.value.status == tps.ERR_INVALID_ARG
