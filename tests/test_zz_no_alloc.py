"""The allocation-free low-rank product (hlu_lowrank_apply_noalloc) against the
library's matrix-vector product.

Some callers may not allocate device memory while they compute, so this entry
point keeps its intermediate in a fixed array inside the library instead of
an arena from hlu_create.  The reference here is hlu_matvec on an H-matrix whose
only non-zero block is one low-rank leaf (U, V): its output rows of that block
are exactly U (V^T x).  Two calls in a row (and a third with a smaller rank)
check that what the shared array kept from the previous call does not leak
into the next result.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1906_00874_gb300 import build, hlu
    build.build()
    lib = hlu.load()
    lib.hlu_lowrank_apply_noalloc.argtypes = [ctypes.c_int32] * 4 + [
        ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
        ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    return lib


def _one_block_hmatrix(U, V):
    """Rows 0..m-1 x columns m..m+n-1 hold U V^T; every other block is zero."""
    from paper_1906_00874_gb300 import HLU
    m, k = U.shape
    n = V.shape[0]
    N = m + n
    begin = np.array([0, 0, m], dtype=np.int32)
    size = np.array([N, m, n], dtype=np.int32)
    son0 = np.array([1, -1, -1], dtype=np.int32)
    son1 = np.array([2, -1, -1], dtype=np.int32)
    rows = np.array([1, 1, 2, 2], dtype=np.int32)
    cols = np.array([1, 2, 1, 2], dtype=np.int32)
    kind = np.array([0, 1, 0, 0], dtype=np.int8)
    rank = np.array([0, k, 0, 0], dtype=np.int32)
    chunks = [np.zeros(m * m), U.ravel(order="F"), V.ravel(order="F"), np.zeros(n * m), np.zeros(n * n)]
    offset = np.array([0, m * m, m * m + (m + n) * k, m * m + (m + n) * k + n * m], dtype=np.int64)
    return HLU(N, np.arange(N), begin, size, son0, son1, rows, cols, kind, rank, offset, np.concatenate(chunks))


def _call(lib, U, V, x_dev, m, n, k, nrhs, row0, ld):
    import torch
    from paper_1906_00874_gb300.hlu import to_device_panel
    Ud, Vd = to_device_panel(U), to_device_panel(V)
    y = torch.full((nrhs, m), 7.0, dtype=torch.float64, device="cuda").t()  # column-major, stale contents
    st = lib.hlu_lowrank_apply_noalloc(m, n, k, nrhs, Ud.data_ptr(), m, Vd.data_ptr(), n,
                                       x_dev.data_ptr() + 8 * row0, ld, y.data_ptr(), m,
                                       torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    return y.cpu().numpy()


def test_noalloc_matches_matvec_on_consecutive_calls(lib):
    import torch
    from paper_1906_00874_gb300.hlu import to_device_panel
    rng = np.random.default_rng(17)
    m, n, nrhs = 100, 90, 5
    for call, k in enumerate((7, 7, 3)):
        U = rng.standard_normal((m, k))
        V = rng.standard_normal((n, k))
        h = _one_block_hmatrix(U, V)
        x = rng.standard_normal((m + n, nrhs))
        xd = to_device_panel(x)
        yd = to_device_panel(np.zeros_like(x))
        h.matvec(xd, yd)  # the library's product (scratch in the handle's arena)
        ref = yd.cpu().numpy()[:m]
        got = _call(lib, U, V, xd, m, n, k, nrhs, row0=m, ld=m + n)
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref)), call
        h.close()
        torch.cuda.synchronize()


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    import torch
    U = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    st = lib.hlu_lowrank_apply_noalloc(1, 1, 300, 300, U.data_ptr(), 1, U.data_ptr(), 1, U.data_ptr(), 1,
                                       U.data_ptr(), 1, None)
    assert st == 1  # HLU_EINVAL: 300 x 300 > 65536


def _ref(U, V, x):
    return U @ (V.T @ x)


@pytest.mark.parametrize("m,n,k,nrhs", [(3001, 2755, 9, 3), (517, 4099, 256, 256), (300, 200, 1, 65536),
                                        (64, 129, 16, 4096)])
def test_noalloc_several_ctas_and_the_largest_accepted_size(lib, m, n, k, nrhs):
    """Several CTAs over the rows (n not a multiple of 128), output tiles with ragged edges and
    k * nrhs at the largest accepted size 65536 (last three cases), against U (V^T x) in
    float64 on the host, on two calls in a row."""
    import torch
    from paper_1906_00874_gb300.hlu import to_device_panel
    rng = np.random.default_rng(m + n + k)
    for _ in range(2):
        U = rng.standard_normal((m, k))
        V = rng.standard_normal((n, k))
        x = rng.standard_normal((n, nrhs))
        xd = to_device_panel(x)
        got = _call(lib, U, V, xd, m, n, k, nrhs, row0=0, ld=n)
        ref = _ref(U, V, x)
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
        torch.cuda.synchronize()


def test_noalloc_rank_zero_clears_y(lib):
    import torch
    m, n, nrhs = 50, 40, 3
    x = torch.ones((nrhs, n), dtype=torch.float64, device="cuda").t()
    y = torch.full((nrhs, m), 7.0, dtype=torch.float64, device="cuda").t()
    st = lib.hlu_lowrank_apply_noalloc(m, n, 0, nrhs, None, m, None, n, x.data_ptr(), n, y.data_ptr(), m,
                                       torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    assert torch.count_nonzero(y).item() == 0


def test_noalloc_rejects_one_past_the_limit(lib):
    import torch
    U = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    st = lib.hlu_lowrank_apply_noalloc(1, 1, 1, 65537, U.data_ptr(), 1, U.data_ptr(), 1, U.data_ptr(), 1,
                                       U.data_ptr(), 1, None)
    assert st == 1  # HLU_EINVAL: 65537 > 65536, rejected before any work is queued
