"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module holds no arithmetic of the block Cimmino method (no scaling, no
A*A^T, no factorisation, no projection).  It only builds the coefficient
matrices, true solutions, right-hand sides f = A*x_true and row-block
partitions of the synthetic workloads.  The paper evaluates on SuiteSparse
matrices (Section 3.3, Table 3.1) that are not available here; these
generators stand in for them:

* ``convdiff2d``  -- 2D convection-diffusion, 5-point first-order upwind
  stencil on an N x N grid (x fastest), h = 1/(N+1), convection b in x.
  Row: diagonal 4 + h*b, west neighbour -1 - h*b, east/north/south -1;
  neighbours outside the grid are dropped (Dirichlet boundary).
* ``convdiff3d``  -- 3D analogue, 7-point upwind stencil on nx*ny*nz
  (x fastest, then y, then z), convection b = (bx, by, bz) >= 0:
  diagonal 6 + h*(bx+by+bz), the upwind neighbour in direction d gets
  -1 - h*b_d, the other neighbours -1.
* ``random_dd``   -- random sparse nonsymmetric matrix: every row has k
  off-diagonal entries in columns drawn uniformly without replacement
  (excluding the diagonal), values N(0,1); the diagonal is
  1.2 * (sum of |off-diagonal|) so A is strictly diagonally dominant.

All matrices are returned as CSR with int64 row pointers, int32 column
indices sorted within each row, and float64 values.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = [
    "CSR", "Workload", "convdiff2d", "convdiff3d", "random_dd",
    "contiguous_blocks", "random_blocks", "uniform_x", "matvec", "workload",
]


@dataclass
class CSR:
    n: int
    row_ptr: np.ndarray   # int64, n+1
    col_idx: np.ndarray   # int32, nnz (sorted within each row)
    val: np.ndarray       # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col_idx] = self.val
        return d


@dataclass
class Workload:
    name: str
    A: CSR
    perm: np.ndarray          # int32, new row r is original row perm[r]
    block_ptr: np.ndarray     # int64, K+1 offsets over permuted rows
    x_true: np.ndarray        # float64, n x nrhs (column-major per RHS: shape (nrhs, n))
    F: np.ndarray             # float64, shape (nrhs, n), F[k] = A @ x_true[k]
    meta: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return len(self.block_ptr) - 1


def _from_triplets(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(n, row_ptr, cols.astype(np.int32), vals.astype(np.float64))


def convdiff2d(N: int, b: float, h: Optional[float] = None) -> CSR:
    """5-point upwind convection-diffusion on an N x N grid, lexicographic (x fastest)."""
    h = 1.0 / (N + 1) if h is None else h
    n = N * N
    r = np.arange(n, dtype=np.int64)
    x = r % N
    y = r // N
    R = [r]; C = [r]; V = [np.full(n, 4.0 + h * b)]
    for mask, off, w in ((x > 0, -1, -1.0 - h * b), (x < N - 1, 1, -1.0),
                         (y > 0, -N, -1.0), (y < N - 1, N, -1.0)):
        R.append(r[mask]); C.append(r[mask] + off); V.append(np.full(int(mask.sum()), w))
    return _from_triplets(n, np.concatenate(R), np.concatenate(C), np.concatenate(V))


def convdiff3d(nx: int, ny: int, nz: int, b, h: Optional[float] = None) -> CSR:
    """7-point upwind convection-diffusion on nx*ny*nz, x fastest then y then z."""
    h = 1.0 / (nx + 1) if h is None else h
    bx, by, bz = (float(t) for t in b)
    n = nx * ny * nz
    r = np.arange(n, dtype=np.int64)
    x = r % nx
    y = (r // nx) % ny
    z = r // (nx * ny)
    R = [r]; C = [r]; V = [np.full(n, 6.0 + h * (bx + by + bz))]
    for coord, ext, stride, bd in ((x, nx, 1, bx), (y, ny, nx, by), (z, nz, nx * ny, bz)):
        lo = coord > 0
        hi = coord < ext - 1
        R.append(r[lo]); C.append(r[lo] - stride); V.append(np.full(int(lo.sum()), -1.0 - h * bd))
        R.append(r[hi]); C.append(r[hi] + stride); V.append(np.full(int(hi.sum()), -1.0))
    return _from_triplets(n, np.concatenate(R), np.concatenate(C), np.concatenate(V))


def random_dd(n: int, k: int, seed: int, dominance: float = 1.2) -> CSR:
    """Random sparse, k off-diagonal N(0,1) entries per row in distinct columns != i,
    diagonal = dominance * row abs-sum of the off-diagonals."""
    rng = np.random.default_rng(seed)
    cols = rng.integers(0, n - 1, size=(n, k), dtype=np.int64)
    rows = np.arange(n, dtype=np.int64)[:, None]
    cols = cols + (cols >= rows)          # skip the diagonal column
    cols.sort(axis=1)
    dup = np.any(cols[:, 1:] == cols[:, :-1], axis=1)
    while dup.any():                      # redraw rows that drew a column twice
        idx = np.nonzero(dup)[0]
        c = rng.integers(0, n - 1, size=(len(idx), k), dtype=np.int64)
        c = c + (c >= idx[:, None])
        c.sort(axis=1)
        cols[idx] = c
        dup = np.any(cols[:, 1:] == cols[:, :-1], axis=1)
    vals = rng.standard_normal(size=(n, k))
    diag = dominance * np.abs(vals).sum(axis=1)
    R = np.concatenate([np.repeat(np.arange(n, dtype=np.int64), k), np.arange(n, dtype=np.int64)])
    C = np.concatenate([cols.ravel(), np.arange(n, dtype=np.int64)])
    V = np.concatenate([vals.ravel(), diag])
    return _from_triplets(n, R, C, V)


def uniform_x(n: int, nrhs: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(nrhs, n))


def matvec(A: CSR, x: np.ndarray) -> np.ndarray:
    """y = A x for building right-hand sides (input construction only)."""
    prod = A.val * x[A.col_idx]
    out = np.zeros(A.n)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    np.add.at(out, rows, prod)
    return out


def contiguous_blocks(n: int, m: int) -> np.ndarray:
    """Uniform (contiguous) partition: blocks of m rows, the last one ragged."""
    bp = list(range(0, n, m)) + [n]
    return np.asarray(bp, dtype=np.int64)


def random_blocks(n: int, lo: int, hi: int, rng: np.random.Generator) -> np.ndarray:
    """Contiguous blocks with m ~ U[lo, hi] until n is covered; a remainder below lo
    merges into the previous block, which is split in two if it then exceeds hi."""
    bp = [0]
    while bp[-1] < n:
        bp.append(min(n, bp[-1] + int(rng.integers(lo, hi + 1))))
    if len(bp) > 2 and bp[-1] - bp[-2] < lo:
        bp.pop(-2)
        last = bp[-1] - bp[-2]
        if last > hi:
            bp.insert(-1, bp[-2] + last // 2)
    return np.asarray(bp, dtype=np.int64)


def _rhs(A: CSR, nrhs: int, seed: int):
    X = uniform_x(A.n, nrhs, seed)
    F = np.stack([matvec(A, X[k]) for k in range(nrhs)])
    return X, F


def workload(cfg: int, scale: str = "full", nrhs: Optional[int] = None) -> Workload:
    """The five synthetic configurations.

    cfg 1: 2D 64x64 (n=4,096), b=20, K=8 contiguous blocks of 512, seed 1.
    cfg 2: 3D 64^3 (n=262,144), b=(30,20,10), K=128 contiguous blocks of 2048, seed 2.
    cfg 3: random n=2^20, 8 off-diagonals/row, K=512 blocks of 2048, seed 3.
    cfg 5: 3D 128^3 (n=2,097,152), b=(50,30,10), K=1024 blocks of 2048, 16 RHS, seed 5.
    ``scale="small"`` shrinks 2/3/5 to a size the oracle finishes in seconds
    (same generator, same block size rule).
    Graph-partitioned variants are built by the partitioner from these inputs.
    """
    if cfg == 1:
        A = convdiff2d(64, 20.0, 1.0 / 65)
        X, F = _rhs(A, nrhs or 1, 1)
        return Workload("convdiff2d_64x64_b20_K8", A, np.arange(A.n, dtype=np.int32),
                        contiguous_blocks(A.n, 512), X, F, {"grid": (64, 64), "seed": 1})
    if cfg == 2:
        N = 64 if scale == "full" else 16
        A = convdiff3d(N, N, N, (30, 20, 10), 1.0 / (N + 1))
        m = 2048 if scale == "full" else 512
        X, F = _rhs(A, nrhs or 1, 2)
        return Workload(f"convdiff3d_{N}^3_b30-20-10_K{A.n // m}", A, np.arange(A.n, dtype=np.int32),
                        contiguous_blocks(A.n, m), X, F, {"grid": (N, N, N), "seed": 2})
    if cfg == 3:
        n = 1 << 20 if scale == "full" else 1 << 14
        A = random_dd(n, 8, 3)
        m = 2048 if scale == "full" else 512
        X, F = _rhs(A, nrhs or 1, 3)
        return Workload(f"random_dd_n{n}_k8_K{n // m}", A, np.arange(n, dtype=np.int32),
                        contiguous_blocks(n, m), X, F, {"seed": 3})
    if cfg == 5:
        N = 128 if scale == "full" else 32
        A = convdiff3d(N, N, N, (50, 30, 10), 1.0 / (N + 1))
        m = 2048 if scale == "full" else 512
        X, F = _rhs(A, nrhs or 16, 5)
        return Workload(f"convdiff3d_{N}^3_b50-30-10_K{A.n // m}_rhs{F.shape[0]}", A,
                        np.arange(A.n, dtype=np.int32), contiguous_blocks(A.n, m), X, F,
                        {"grid": (N, N, N), "seed": 5})
    raise ValueError(f"unknown config {cfg}")


def batch_workload(nsys: int = 64, seed: int = 4, max_nz: int = 64):
    """Config 4: nsys independent 3D convection-diffusion systems on 64x64xnz grids,
    nz = round(exp(U[ln 4, ln max_nz])), b ~ U[5,40]^3, blocks m ~ U[256, 2048]."""
    rng = np.random.default_rng(seed)
    out: List[Workload] = []
    for s in range(nsys):
        nz = int(round(np.exp(rng.uniform(np.log(4), np.log(max_nz)))))
        b = rng.uniform(5, 40, size=3)
        A = convdiff3d(64, 64, nz, b, 1.0 / 65)
        bp = random_blocks(A.n, 256, 2048, rng)
        X = rng.uniform(-1.0, 1.0, size=(1, A.n))
        F = matvec(A, X[0])[None, :]
        out.append(Workload(f"sys{s}_64x64x{nz}", A, np.arange(A.n, dtype=np.int32), bp, X, F,
                            {"grid": (64, 64, nz), "b": tuple(b)}))
    return out
