"""Plain FP64 CPU oracle of the CG-accelerated block Cimmino solve (arXiv 1710.07769).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline / reference leg of ``bench.py``.  The product package
never imports it.  The arithmetic lives in ``cimmino_oracle.c`` (plain loops,
FP64, no floating-point contraction); this module only builds that file with
gcc and marshals arguments through ctypes.

Functions and the paper passages they follow:
  * ``Oracle(..., ruiz=k)``: k sweeps of row and column infinity-norm
    equilibration first (Section 3.1; ``equil()`` returns the factors), then
    row 2-norm prescaling (Section 2.1), row permutation
    A^Pi = P A (Section 2.2), C = A A^T by Gustavson SpGEMM (Section 2.3),
    Gram blocks G_i = A_i A_i^T and their Cholesky factors (the pseudoinverse
    A_i^+ = A_i^T (A_i A_i^T)^{-1} of Section 1, applied, never formed).
  * ``Oracle.project``: H v = sum_i A_i^+ A_i v (Eq. 1.5).
  * ``Oracle.project_rhs``: xi = sum_i A_i^+ f_i (Section 1.1).
  * ``Oracle.solve``: Algorithm 2 from x^(0) = 0 (Section 3.1), stopping on the
    true relative residual; gamma of Eq. 3.1 is reported too.
  * ``Oracle.cimmino_sweeps``: Algorithm 1 with relaxation omega.
  * ``cutsize`` / ``ip_matrix``: Eqs. 2.6-2.9.
  * ``sparsify_dense_columns``: the dense-column rule of Section 2.3 (the graph
    is built from a copy of A whose dense columns keep their sqrt(n) largest
    entries).
  * ``aat_plain`` / ``cholesky_dense``: the same SpGEMM / Cholesky code on a
    caller matrix, for pins against independent references.
Parity status of every function is pinned by ``tests/test_oracle_pins.py``; the
paper's own worked example (Figures 2.1-2.5) is unpinned beyond the single
inner product it prints, because its matrix exists only in a figure.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cimmino_oracle.c")
_LIB = os.path.join(_HERE, "libcimmino_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_ESINGULAR, ORC_ENOCONV, ORC_EBREAKDOWN = 0, -1, -2, -3, -4, -5

_p = C.c_void_p
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -ffp-contract=off, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        lib.orc_setup.argtypes = [C.c_int64, _i64p, _i32p, _f64p, C.c_int32, _i32p, _i64p,
                                  C.c_int32, C.c_int, C.c_int, C.POINTER(_p)]
        lib.orc_setup.restype = C.c_int
        lib.orc_free.argtypes = [_p]
        lib.orc_fail_block.argtypes = [_p]
        lib.orc_fail_block.restype = C.c_int32
        lib.orc_aat_nnz.argtypes = [_p]
        lib.orc_aat_nnz.restype = C.c_int64
        lib.orc_aat_get.argtypes = [_p, _i64p, _i32p, _f64p]
        lib.orc_scaled_get.argtypes = [_p, _i64p, _i32p, _f64p, _f64p]
        lib.orc_equil_get.argtypes = [_p, _f64p, _f64p]
        lib.orc_factor_get.argtypes = [_p, C.c_int32, _f64p]
        lib.orc_gram_get.argtypes = [_p, C.c_int32, _f64p]
        lib.orc_project.argtypes = [_p, _f64p, _f64p]
        lib.orc_project_rhs.argtypes = [_p, _f64p, _f64p]
        lib.orc_solve.argtypes = [_p, _f64p, C.c_double, C.c_int32, _f64p, C.POINTER(C.c_int32),
                                  C.POINTER(C.c_double), C.POINTER(C.c_double), _p]
        lib.orc_solve.restype = C.c_int
        lib.orc_cimmino_sweeps.argtypes = [_p, _f64p, C.c_double, C.c_int32, _f64p]
        lib.orc_cutsize.argtypes = [C.c_int64, _i64p, _i32p, _f64p, _i32p]
        lib.orc_cutsize.restype = C.c_double
        lib.orc_ip_matrix.argtypes = [C.c_int64, _i64p, _i32p, _f64p, _i32p, C.c_int32, _f64p]
        lib.orc_aat_plain.argtypes = [C.c_int64, _i64p, _i32p, _f64p, _p, _p, _p,
                                      C.POINTER(C.c_int64)]
        lib.orc_aat_plain.restype = C.c_int
        lib.orc_sparsify_dense_columns.argtypes = [C.c_int64, _i64p, _i32p, _f64p, _i64p,
                                                   _i32p, _f64p]
        lib.orc_sparsify_dense_columns.restype = C.c_int64
        lib.orc_cholesky_dense.argtypes = [C.c_int64, _f64p]
        lib.orc_cholesky_dense.restype = C.c_int
        lib.orc_factor_range.argtypes = [_p, C.c_int32, C.c_int32]
        lib.orc_factor_range.restype = C.c_int
        lib.orc_solve_range.argtypes = [_p, _f64p, _f64p]
        lib.orc_solve_range.restype = C.c_int
        _lib = lib
        return lib


class OracleError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class Oracle:
    """Setup of the FP64 oracle for one system and one row-block partition."""

    def __init__(self, A, block_ptr, perm=None, factor: bool = True, nthreads: int = 1,
                 ruiz: int = 0):
        lib = _load()
        self.lib = lib
        self.n = int(A.n)
        self.block_ptr = np.ascontiguousarray(block_ptr, dtype=np.int64)
        self.K = len(self.block_ptr) - 1
        perm = np.arange(self.n, dtype=np.int32) if perm is None else perm
        self.perm = np.ascontiguousarray(perm, dtype=np.int32)
        self._A = (np.ascontiguousarray(A.row_ptr, dtype=np.int64),
                   np.ascontiguousarray(A.col_idx, dtype=np.int32),
                   np.ascontiguousarray(A.val, dtype=np.float64))
        h = _p()
        self.ruiz = int(ruiz)
        st = lib.orc_setup(self.n, *self._A, self.K, self.perm, self.block_ptr, self.ruiz,
                           int(factor), int(nthreads), C.byref(h))
        self._h = h
        if st != ORC_OK:
            fb = lib.orc_fail_block(h) if h.value else -1
            self.close()
            raise OracleError(st, f"oracle setup failed (block {fb})")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.orc_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- accessors -------------------------------------------------------
    def aat(self):
        nnz = self.lib.orc_aat_nnz(self._h)
        rp = np.zeros(self.n + 1, np.int64)
        ci = np.zeros(max(nnz, 1), np.int32)
        v = np.zeros(max(nnz, 1), np.float64)
        self.lib.orc_aat_get(self._h, rp, ci, v)
        return rp, ci[:nnz], v[:nnz]

    def scaled(self):
        nnz = int(self._A[0][-1])
        rp = np.zeros(self.n + 1, np.int64)
        ci = np.zeros(max(nnz, 1), np.int32)
        v = np.zeros(max(nnz, 1), np.float64)
        d = np.zeros(self.n, np.float64)
        self.lib.orc_scaled_get(self._h, rp, ci, v, d)
        return rp, ci[:nnz], v[:nnz], d

    def equil(self):
        """(rs, cs) with A = diag(rs) Ae diag(cs), Ae the equilibrated matrix."""
        rs = np.zeros(self.n, np.float64)
        cs = np.zeros(self.n, np.float64)
        self.lib.orc_equil_get(self._h, rs, cs)
        return rs, cs

    def block_size(self, b: int) -> int:
        return int(self.block_ptr[b + 1] - self.block_ptr[b])

    def factor(self, b: int) -> np.ndarray:
        m = self.block_size(b)
        L = np.zeros(m * m)
        self.lib.orc_factor_get(self._h, int(b), L)
        return L.reshape(m, m)

    def gram(self, b: int) -> np.ndarray:
        m = self.block_size(b)
        G = np.zeros(m * m)
        self.lib.orc_gram_get(self._h, int(b), G)
        return G.reshape(m, m)

    def factor_range(self, b0: int, b1: int) -> int:
        """Cholesky of the Gram blocks [b0, b1) only (the full setup's routine, into
        storage of their own): a bounded sample of the factorisation.  Returns the status."""
        return int(self.lib.orc_factor_range(self._h, int(b0), int(b1)))

    def solve_range(self, u: np.ndarray) -> np.ndarray:
        """y_i = G_i^{-1} u_i for the blocks of the last factor_range (permuted-row
        n-vectors; other rows of y stay zero): a bounded sample of a projection's solves."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        y = np.zeros(self.n)
        st = self.lib.orc_solve_range(self._h, u, y)
        if st != ORC_OK:
            raise OracleError(st, "solve_range needs a factor_range first")
        return y

    # --- the method ---------------------------------------------------------
    def project(self, v: np.ndarray) -> np.ndarray:
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(self.n)
        self.lib.orc_project(self._h, v, out)
        return out

    def project_rhs(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros(self.n)
        self.lib.orc_project_rhs(self._h, f, out)
        return out

    def solve(self, f: np.ndarray, tol: float = 1e-10, maxit: int = 10000, history: bool = False):
        """Algorithm 2.  Returns (x, iters, relres, gamma, status[, hist])."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        x = np.zeros(self.n)
        it = C.c_int32(0)
        rr = C.c_double(0.0)
        g = C.c_double(0.0)
        hist = np.zeros(max(maxit, 1)) if history else None
        st = self.lib.orc_solve(self._h, f, float(tol), int(maxit), x, C.byref(it), C.byref(rr),
                                C.byref(g), hist.ctypes.data_as(_p) if history else None)
        out = (x, int(it.value), float(rr.value), float(g.value), int(st))
        return out + (hist[: it.value],) if history else out

    def cimmino_sweeps(self, f: np.ndarray, omega: float, sweeps: int) -> np.ndarray:
        """Algorithm 1 (block Cimmino with relaxation omega) from x^(0) = 0."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        x = np.zeros(self.n)
        self.lib.orc_cimmino_sweeps(self._h, f, float(omega), int(sweeps), x)
        return x


def cutsize(Crp, Cci, Cv, part) -> float:
    """cutsize(Pi) = interIP(Pi), Eqs. 2.6-2.7 (each undirected edge counted once)."""
    lib = _load()
    return float(lib.orc_cutsize(len(Crp) - 1, np.ascontiguousarray(Crp, np.int64),
                                 np.ascontiguousarray(Cci, np.int32),
                                 np.ascontiguousarray(Cv, np.float64),
                                 np.ascontiguousarray(part, np.int32)))


def ip_matrix(Crp, Cci, Cv, part, K: int) -> np.ndarray:
    """ip_km of Eqs. 2.8-2.9 (K x K; off-diagonal entries are the inter-block sums)."""
    lib = _load()
    out = np.zeros(K * K)
    lib.orc_ip_matrix(len(Crp) - 1, np.ascontiguousarray(Crp, np.int64),
                      np.ascontiguousarray(Cci, np.int32), np.ascontiguousarray(Cv, np.float64),
                      np.ascontiguousarray(part, np.int32), int(K), out)
    return out.reshape(K, K)


def sparsify_dense_columns(A):
    """(row_ptr, col_idx, val) of A with every dense column (more than floor(sqrt(n))
    nonzeros) cut to its floor(sqrt(n)) largest magnitudes (Section 2.3)."""
    lib = _load()
    rp, ci, v = (np.ascontiguousarray(A.row_ptr, np.int64), np.ascontiguousarray(A.col_idx, np.int32),
                 np.ascontiguousarray(A.val, np.float64))
    nnz = int(rp[-1])
    orp = np.zeros(A.n + 1, np.int64)
    oci = np.zeros(max(nnz, 1), np.int32)
    ov = np.zeros(max(nnz, 1), np.float64)
    w = lib.orc_sparsify_dense_columns(A.n, rp, ci, v, orp, oci, ov)
    return orp, oci[:w], ov[:w]


def aat_plain(A):
    """C = A A^T of a caller matrix (no scaling / permutation), Gustavson, structural pattern."""
    lib = _load()
    rp, ci, v = (np.ascontiguousarray(A.row_ptr, np.int64), np.ascontiguousarray(A.col_idx, np.int32),
                 np.ascontiguousarray(A.val, np.float64))
    nnz = C.c_int64(0)
    crp = np.zeros(A.n + 1, np.int64)
    st = lib.orc_aat_plain(A.n, rp, ci, v, crp.ctypes.data_as(_p), None, None, C.byref(nnz))
    if st != ORC_OK:
        raise OracleError(st, "aat failed")
    cci = np.zeros(max(nnz.value, 1), np.int32)
    cv = np.zeros(max(nnz.value, 1), np.float64)
    lib.orc_aat_plain(A.n, rp, ci, v, crp.ctypes.data_as(_p), cci.ctypes.data_as(_p),
                      cv.ctypes.data_as(_p), C.byref(nnz))
    return crp, cci[: nnz.value], cv[: nnz.value]


def cholesky_dense(G: np.ndarray):
    """Lower Cholesky factor of a dense SPD matrix with the oracle's code; (L, status)."""
    m = G.shape[0]
    a = np.ascontiguousarray(G, dtype=np.float64).copy().ravel()
    st = _load().orc_cholesky_dense(m, a)
    return a.reshape(m, m), int(st)
