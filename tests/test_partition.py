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
