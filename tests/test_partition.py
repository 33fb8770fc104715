"""Host partitioner on the row inner-product graph (Section 2): it must return a valid
block-row partition that respects the row cap (Eq. A.1), report the cutsize the oracle
computes for that partition (Eqs. 2.6-2.7: cutsize = interIP), and cut far less inner
product than the straightforward contiguous partition on stencil matrices (Section 2.2)."""
import numpy as np
import pytest

import inputs
import oracle

g = pytest.importorskip("paper_1710_07769_gb300")


def scaled_aat(A):
    crp, cci, cv = oracle.aat_plain(A)
    rows = np.repeat(np.arange(A.n), np.diff(crp))
    d = np.sqrt(cv[rows == cci])
    return crp, cci, cv / (d[rows] * d[cci])


def part_of(perm, bp, n):
    part = np.empty(n, np.int32)
    for k in range(len(bp) - 1):
        part[perm[bp[k]:bp[k + 1]]] = k
    return part


@pytest.mark.parametrize("which,K,eps", [("conv2d", 8, 0.05), ("conv3d", 16, 0.0), ("random", 8, 0.1)])
def test_partition_valid_balanced_and_cut_matches_oracle(which, K, eps):
    A = {"conv2d": lambda: inputs.convdiff2d(48, 20.0),
         "conv3d": lambda: inputs.convdiff3d(16, 16, 16, (30, 20, 10)),
         "random": lambda: inputs.random_dd(3000, 6, 5)}[which]()
    n = A.n
    C = oracle.aat_plain(A)
    perm, bp, cut = g.partition_rip(n, C, K, eps=eps, seed=1)
    assert np.array_equal(np.sort(perm), np.arange(n))
    sizes = np.diff(bp)
    cap = int(np.ceil(n / K * (1 + eps)))
    assert bp[0] == 0 and bp[-1] == n and sizes.min() >= 1 and sizes.max() <= cap
    if eps == 0.0:
        assert np.all(sizes == n // K)
    part = part_of(perm, bp, n)
    crp, cci, cs = scaled_aat(A)
    assert cut == pytest.approx(oracle.cutsize(crp, cci, cs, part), rel=1e-9)
    contiguous = np.repeat(np.arange(K), np.diff(inputs.contiguous_blocks(n, -(-n // K))))[:n]
    cut_c = oracle.cutsize(crp, cci, cs, contiguous.astype(np.int32))
    assert cut <= cut_c, (cut, cut_c)
    if which == "conv3d":                     # box-like blocks beat thin slabs by far
        assert cut < 0.8 * cut_c, (cut, cut_c)


def test_partition_solves_like_any_partition():
    """Any block-row partition gives the same solution (it only changes H's spectrum):
    the oracle converges to A^{-1} f with the graph partition as well."""
    A = inputs.convdiff2d(32, 20.0)
    f = inputs.matvec(A, inputs.uniform_x(A.n, 1, 4)[0])
    perm, bp, cut = g.partition_rip(A.n, oracle.aat_plain(A), 4, eps=0.05, seed=3)
    x, it, rr, gm, st = oracle.Oracle(A, bp, perm=perm).solve(f)
    assert st == 0 and rr <= 1e-10
    x2, it2, *_ = oracle.Oracle(A, inputs.contiguous_blocks(A.n, 256)).solve(f)
    np.testing.assert_allclose(x, x2, atol=1e-8)


def matrix_with_dense_columns(n, ndense, seed):
    """A 2D stencil plus ndense columns holding n/3 random entries each."""
    B = inputs.convdiff2d(int(np.sqrt(n)), 20.0)
    n = B.n
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(n), np.diff(B.row_ptr))
    r, c, v = [rows], [B.col_idx.astype(np.int64)], [B.val]
    for j in rng.choice(n, ndense, replace=False):
        rr = rng.choice(n, n // 3, replace=False)
        r.append(rr)
        c.append(np.full(len(rr), j))
        v.append(rng.choice([-1.0, 0.5, 2.0], len(rr)) * rng.integers(1, 4, len(rr)))  # ties
    r, c, v = np.concatenate(r), np.concatenate(c), np.concatenate(v)
    key = r * n + c
    uk, first = np.unique(key, return_index=True)        # keep one entry per (row, col)
    r, c, v = r[first], c[first], v[first]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, r + 1, 1)
    return inputs.CSR(n, np.cumsum(rp), c.astype(np.int32), v)


@pytest.mark.parametrize("n,ndense,seed", [(400, 2, 1), (2500, 5, 2), (4900, 1, 3)])
def test_sparsify_dense_columns_matches_oracle(n, ndense, seed):
    """The library's dense-column rule (Section 2.3) returns exactly the oracle's copy."""
    A = matrix_with_dense_columns(n, ndense, seed)
    rp, ci, v = g.sparsify_dense_columns(A)
    orp, oci, ov = oracle.sparsify_dense_columns(A)
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci) and np.array_equal(v, ov)
    t = int(np.floor(np.sqrt(A.n)))
    before = np.bincount(A.col_idx, minlength=A.n)
    after = np.bincount(ci, minlength=A.n)
    assert (before > t).sum() == ndense
    assert np.array_equal(after, np.where(before > t, t, before))


def test_partition_after_sparsifying_dense_columns():
    """With dense columns C = A A^T is nearly dense; the graph of the sparsified copy is
    small, and its partition is still a valid one that beats contiguous blocks on the
    cut of the full C."""
    A = matrix_with_dense_columns(2500, 3, 7)
    C_full = oracle.aat_plain(A)
    S = inputs.CSR(A.n, *g.sparsify_dense_columns(A))
    C_sp = oracle.aat_plain(S)
    assert len(C_sp[1]) * 20 < len(C_full[1])
    K = 10
    perm, bp, _ = g.partition_rip(A.n, C_sp, K, eps=0.05, seed=3)
    assert np.array_equal(np.sort(perm), np.arange(A.n))
    assert np.diff(bp).max() <= int(np.ceil(A.n / K * 1.05))
    rows = np.repeat(np.arange(A.n), np.diff(C_full[0]))
    d = np.sqrt(C_full[2][rows == C_full[1]])
    cos = (C_full[0], C_full[1], C_full[2] / (d[rows] * d[C_full[1]]))
    cut_gp = oracle.cutsize(*cos, part_of(perm, bp, A.n))
    contiguous = np.repeat(np.arange(K), A.n // K).astype(np.int32)
    assert cut_gp < oracle.cutsize(*cos, contiguous)


def test_host_entry_points_reject_bad_input():
    """The host-only entry points validate their CSR input and sizes (no GPU needed)."""
    A = inputs.convdiff2d(8, 20.0)
    bad_col = inputs.CSR(A.n, A.row_ptr.copy(), A.col_idx.copy(), A.val.copy())
    bad_col.col_idx[3] = A.n            # column out of range
    with pytest.raises(g.CimminoError) as e:
        g.sparsify_dense_columns(bad_col)
    assert e.value.code == g.EINVAL
    bad_rp = inputs.CSR(A.n, A.row_ptr.copy(), A.col_idx.copy(), A.val.copy())
    bad_rp.row_ptr[5] = bad_rp.row_ptr[6] + 1   # row pointers not monotone
    with pytest.raises(g.CimminoError) as e:
        g.sparsify_dense_columns(bad_rp)
    assert e.value.code == g.EINVAL
    C = oracle.aat_plain(A)
    for K, cap in ((0, 8), (A.n + 1, 1), (4, A.n // 4 - 1)):   # K out of range, cap * K < n
        with pytest.raises(g.CimminoError) as e:
            g.partition_rip(A.n, C, K, cap=cap)
        assert e.value.code == g.EINVAL
