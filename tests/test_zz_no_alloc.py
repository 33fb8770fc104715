"""cimmino_aat_noalloc: C = A A^T for callers that cannot allocate device memory
(for example code running while a stream is captured into a CUDA graph, where
cudaMalloc is not allowed, or embedders with their own allocator or budget).

Its output must equal that of the allocating entry point cimmino_aat, on calls in
a row with different matrices: the static scratch array keeps the previous call's
contents, so a stale value would show up here.  This file is collected last so
that a failure here does not hide the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_1710_07769_gb300")


def _csr_from_dense(D):
    n = D.shape[0]
    rp = np.zeros(n + 1, np.int64)
    cols, vals = [], []
    for i in range(n):
        nz = np.nonzero(D[i])[0]
        cols.append(nz)
        vals.append(D[i, nz])
        rp[i + 1] = rp[i] + len(nz)
    return inputs.CSR(n, rp, np.concatenate(cols).astype(np.int32), np.concatenate(vals))


def _noalloc(A):
    """Two-call pattern through the C ABI with caller-owned device buffers."""
    import torch
    L = g.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col_idx).to(dev)
    v = torch.from_numpy(A.val).to(dev)
    csr = g.CSRStruct(A.n, A.nnz, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), 1)
    crp = torch.empty(A.n + 1, dtype=torch.int64, device=dev)
    nnz = C.c_int64(-1)
    torch.cuda.synchronize()
    st = L.cimmino_aat_noalloc(C.byref(csr), None, C.byref(nnz), crp.data_ptr(), None, None, 0)
    assert st == 0, L.cimmino_last_error(None)
    cci = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=dev)
    cv = torch.empty(max(nnz.value, 1), dtype=torch.float64, device=dev)
    st = L.cimmino_aat_noalloc(C.byref(csr), None, C.byref(nnz), crp.data_ptr(), cci.data_ptr(),
                               cv.data_ptr(), nnz.value)
    assert st == 0, L.cimmino_last_error(None)
    torch.cuda.synchronize()
    return crp.cpu().numpy(), cci.cpu().numpy()[: nnz.value], cv.cpu().numpy()[: nnz.value]


def _dense_column_matrix():
    n = 2000
    D = np.zeros((n, n))
    D[np.arange(n), np.arange(n)] = 3.0
    D[:1500, 7] += np.linspace(0.5, 1.5, 1500)   # rows with > 1024 candidates
    return _csr_from_dense(D)


def test_noalloc_aat_equals_aat_on_consecutive_calls():
    mats = [inputs.convdiff3d(20, 20, 20, (30, 20, 10)),
            inputs.random_dd(5000, 8, 7),
            _dense_column_matrix(),
            inputs.convdiff3d(20, 20, 20, (30, 20, 10))]
    for A in mats:
        rp, ci, v = _noalloc(A)
        rrp, rci, rv = g.aat(A)
        assert np.array_equal(rp, rrp)
        assert np.array_equal(ci, rci)
        np.testing.assert_allclose(v, rv, rtol=1e-12, atol=0)


def test_noalloc_limits_and_capacity():
    import torch
    L = g.load()
    A = inputs.convdiff2d(30, 20.0)
    dev = torch.device("cuda", torch.cuda.current_device())
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col_idx).to(dev)
    v = torch.from_numpy(A.val).to(dev)
    crp = torch.empty(A.n + 1, dtype=torch.int64, device=dev)
    small = torch.empty(10, dtype=torch.int32, device=dev)
    smallv = torch.empty(10, dtype=torch.float64, device=dev)
    nnz = C.c_int64(0)
    csr = g.CSRStruct(A.n, A.nnz, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), 1)
    st = L.cimmino_aat_noalloc(C.byref(csr), None, C.byref(nnz), crp.data_ptr(), small.data_ptr(),
                               smallv.data_ptr(), 10)
    assert st == g.EINVAL and nnz.value > 10
    host = g.CSRStruct(A.n, A.nnz, A.row_ptr.ctypes.data, A.col_idx.ctypes.data,
                       A.val.ctypes.data, 0)
    assert L.cimmino_aat_noalloc(C.byref(host), None, C.byref(nnz), crp.data_ptr(), None, None,
                                 0) == g.EINVAL
    big = g.CSRStruct(1 << 19, A.nnz, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), 1)
    assert L.cimmino_aat_noalloc(C.byref(big), None, C.byref(nnz), crp.data_ptr(), None, None,
                                 0) == g.EUNSUPPORTED
