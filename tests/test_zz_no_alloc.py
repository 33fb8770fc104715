"""cimmino_aat_noalloc: C = A A^T for callers that cannot let a library allocate device
memory (embedders whose device memory is reserved by their own caching allocator or capped
by a fixed budget, and latency-bound loops that cannot afford cudaMalloc / cudaFree).

Its output must equal that of the allocating entry point cimmino_aat, and the oracle's
plain Gustavson product, on calls in a row with different matrices: the static scratch
array keeps the previous call's contents, so a stale value would show up here.  A call
that is rejected half-way (a row of A A^T with too many candidates) must not spoil the
next one.  This file is collected last so that a failure here does not hide the other
GPU tests.
"""
import ctypes as C

import numpy as np
import pytest

import inputs
import oracle

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
        # and the oracle's plain product (Section 2.3): same structural pattern, values to
        # 1e-12 relative of the row's largest magnitude
        orp, oci, ov = oracle.aat_plain(A)
        assert np.array_equal(rp, orp) and np.array_equal(ci, oci)
        rowmax = np.maximum.reduceat(np.abs(ov), orp[:-1]) if len(ov) else ov
        scale = np.repeat(rowmax, np.diff(orp))
        assert np.all(np.abs(v - ov) <= 1e-12 * scale)


def _last_error():
    return g.load().cimmino_last_error(None).decode()


def test_noalloc_rejected_call_then_clean_call():
    """A count that fails half-way (a row of A A^T with more than 8192 structural
    candidates: 9000 rows share one column) returns EUNSUPPORTED with its message; the next
    call on another matrix must still equal cimmino_aat (flags and counts start clean)."""
    import torch
    L = g.load()
    n = 12000
    D_rows = np.arange(n)
    rp = np.zeros(n + 1, np.int64)
    cols, vals = [], []
    for i in D_rows:
        c = [i] if i >= 9000 or i == 5 else sorted({5, int(i)})
        cols.append(np.array(c, np.int32))
        vals.append(np.where(np.array(c) == i, 3.0, 1.0 + 1e-4 * i))
        rp[i + 1] = rp[i] + len(c)
    bad = inputs.CSR(n, rp, np.concatenate(cols), np.concatenate(vals))
    dev = torch.device("cuda", torch.cuda.current_device())
    drp = torch.from_numpy(bad.row_ptr).to(dev)
    dci = torch.from_numpy(bad.col_idx).to(dev)
    dv = torch.from_numpy(bad.val).to(dev)
    csr = g.CSRStruct(bad.n, bad.nnz, drp.data_ptr(), dci.data_ptr(), dv.data_ptr(), 1)
    crp = torch.empty(bad.n + 1, dtype=torch.int64, device=dev)
    nnz = C.c_int64(0)
    st = L.cimmino_aat_noalloc(C.byref(csr), None, C.byref(nnz), crp.data_ptr(), None, None, 0)
    assert st == g.EUNSUPPORTED, st
    assert "8192" in _last_error()
    for A in (inputs.convdiff3d(20, 20, 20, (30, 20, 10)), _dense_column_matrix()):
        rp2, ci2, v2 = _noalloc(A)
        rrp, rci, rv = g.aat(A)
        assert np.array_equal(rp2, rrp) and np.array_equal(ci2, rci)
        np.testing.assert_allclose(v2, rv, rtol=1e-12, atol=0)


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
    assert "capacity" in _last_error()
    host = g.CSRStruct(A.n, A.nnz, A.row_ptr.ctypes.data, A.col_idx.ctypes.data,
                       A.val.ctypes.data, 0)
    assert L.cimmino_aat_noalloc(C.byref(host), None, C.byref(nnz), crp.data_ptr(), None, None,
                                 0) == g.EINVAL
    assert "device memory" in _last_error()
    big = g.CSRStruct(1 << 19, A.nnz, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), 1)
    assert L.cimmino_aat_noalloc(C.byref(big), None, C.byref(nnz), crp.data_ptr(), None, None,
                                 0) == g.EUNSUPPORTED
    assert "262144" in _last_error()
