"""Python binding of libcimmino.so, the GB300 (sm_103a) CG-accelerated block Cimmino solver.

The library (C ABI in ``include/cimmino.h``) runs Algorithm 2 of Torun, Manguoglu
and Aykanat (arXiv 1710.07769): classical CG on H x = xi with
H = sum_i A_i^T (A_i A_i^T)^{-1} A_i over the K block rows A_i of A.  This module
only marshals arguments: every step of the computation runs in the library's
CUDA kernels.  Host inputs are numpy arrays; device inputs are torch CUDA
tensors (torch supplies device memory and the stream).  There is no CPU
fallback: a missing library raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

__all__ = ["FP64", "FP32_REFINE", "DENSE", "SKYLINE", "CimminoError", "Solver", "BatchSolver",
           "aat", "partition_rip", "sparsify_dense_columns", "cholesky_schedule", "selftest_wait",
           "fp64_peak", "load",
           "lib_path", "EXPORTS"]

FP64, FP32_REFINE = 0, 1
DENSE, SKYLINE = 0, 1
OK, EINVAL, ENOMEM, ESINGULAR, ENOCONV, EBREAKDOWN, ETIMEOUT, ECUDA, EUNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ESINGULAR", -4: "ENOCONV", -5: "EBREAKDOWN",
          -6: "ETIMEOUT", -7: "ECUDA", -8: "EUNSUPPORTED"}

# every entry point declared in include/cimmino.h
EXPORTS = ["cimmino_opts_default", "cimmino_setup", "cimmino_setup_batch", "cimmino_solve",
           "cimmino_solve_batch", "cimmino_free", "cimmino_last_error", "cimmino_get_aat_nnz",
           "cimmino_get_aat", "cimmino_get_scaled", "cimmino_get_colscale", "cimmino_block_rows", "cimmino_get_factor",
           "cimmino_project", "cimmino_project_rhs", "cimmino_sweeps", "cimmino_aat",
           "cimmino_aat_noalloc",
           "cimmino_partition_rip", "cimmino_sparsify_dense_columns", "cimmino_proj_timing",
           "cimmino_selftest_wait", "cimmino_time_kernels", "cimmino_fp64_peak",
           "cimmino_cholesky_schedule", "cimmino_version"]


class CSRStruct(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p), ("on_device", C.c_int32)]


# caller device allocator of a context (cimmino_opts.alloc / .free)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class OptsStruct(C.Structure):
    _fields_ = [("precision", C.c_int32), ("layout", C.c_int32), ("tile", C.c_int32),
                ("refine_max", C.c_int32), ("refine_tol", C.c_double),
                ("pivot_ratio_min", C.c_double), ("max_iter", C.c_int32),
                ("use_graph", C.c_int32), ("check_every", C.c_int32), ("keep_aat", C.c_int32),
                ("refine_relax", C.c_int32), ("multi_rhs", C.c_int32),
                ("ruiz_sweeps", C.c_int32), ("time_proj", C.c_int32), ("stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
                ("tune", C.c_int32), ("tune_cache", C.c_char_p)]


def torch_allocator():
    """(alloc, free) callbacks that take a context's device memory from torch's caching
    allocator on the context's stream.  Keep the returned objects alive as long as the
    context (the Solver classes do)."""
    import torch

    dev = torch.cuda.current_device()

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass

    return ALLOC_FN(_alloc), FREE_FN(_free)


class StatsStruct(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("rel_res", C.c_double),
                ("backward_err", C.c_double), ("refine_steps_total", C.c_int64),
                ("refine_steps_max", C.c_int32), ("fallbacks", C.c_int32),
                ("t_setup_ms", C.c_double), ("t_factor_ms", C.c_double),
                ("t_solve_ms", C.c_double), ("nnz_aat", C.c_int64), ("factor_bytes", C.c_int64),
                ("pass_bytes", C.c_int64), ("kernel_launches", C.c_int64),
                ("factor_flops", C.c_double), ("t_chol_ms", C.c_double),
                ("nnz_gram", C.c_int64), ("proj_slots", C.c_int32),
                ("proj_ctas_per_sm", C.c_int32), ("proj_tuned", C.c_int32),
                ("mr_tc_blocks", C.c_int32), ("chol_split_blocks", C.c_int32)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = _NAMES.get(self.status, str(self.status))
        return d


class CimminoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.OUT


def load(build_if_missing: bool = False):
    """Load libcimmino.so (raises RuntimeError when it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is not built; run paper_1710_07769_gb300.build.build()")
            _build.build()
        L = C.CDLL(path)
        vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.cimmino_opts_default.argtypes = [C.POINTER(OptsStruct)]
        L.cimmino_setup.argtypes = [C.POINTER(CSRStruct), i32, vp, vp, C.POINTER(OptsStruct),
                                    C.POINTER(vp)]
        L.cimmino_setup_batch.argtypes = [i32, C.POINTER(CSRStruct), vp, vp, vp,
                                          C.POINTER(OptsStruct), C.POINTER(vp)]
        L.cimmino_solve.argtypes = [vp, vp, i32, i64, dbl, vp, i32, C.POINTER(StatsStruct)]
        L.cimmino_solve_batch.argtypes = [vp, vp, dbl, vp, i32, C.POINTER(StatsStruct)]
        L.cimmino_free.argtypes = [vp]
        L.cimmino_free.restype = None
        L.cimmino_last_error.argtypes = [vp]
        L.cimmino_last_error.restype = C.c_char_p
        L.cimmino_get_aat_nnz.argtypes = [vp, C.POINTER(i64)]
        L.cimmino_get_aat.argtypes = [vp, vp, vp, vp]
        L.cimmino_get_scaled.argtypes = [vp, vp, vp, vp, vp]
        L.cimmino_get_colscale.argtypes = [vp, vp]
        L.cimmino_block_rows.argtypes = [vp, i32, C.POINTER(i32)]
        L.cimmino_get_factor.argtypes = [vp, i32, vp, C.POINTER(i32)]
        L.cimmino_project.argtypes = [vp, vp, i32, vp, i32]
        L.cimmino_project_rhs.argtypes = [vp, vp, i32, vp, i32]
        L.cimmino_sweeps.argtypes = [vp, vp, i32, dbl, i32, vp, i32]
        L.cimmino_aat.argtypes = [C.POINTER(CSRStruct), vp, C.POINTER(i64), vp, vp, vp]
        L.cimmino_time_kernels.argtypes = [vp, i32, vp]
        L.cimmino_proj_timing.argtypes = [vp, C.POINTER(dbl), C.POINTER(i64)]
        L.cimmino_selftest_wait.argtypes = [i32, C.POINTER(i32)]
        L.cimmino_fp64_peak.argtypes = [C.POINTER(dbl)]
        L.cimmino_partition_rip.argtypes = [i64, vp, vp, vp, i32, i32, C.c_uint64, vp, vp,
                                            C.POINTER(dbl)]
        L.cimmino_sparsify_dense_columns.argtypes = [i64, vp, vp, vp, vp, vp, vp,
                                                     C.POINTER(i64)]
        L.cimmino_aat_noalloc.argtypes = [C.POINTER(CSRStruct), vp, C.POINTER(i64), vp, vp, vp, i64]
        L.cimmino_cholesky_schedule.argtypes = [i32, vp, vp, vp, i32, i32, C.POINTER(i32), vp, vp,
                                                C.POINTER(i32), C.POINTER(dbl)]
        L.cimmino_version.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("cimmino_free", "cimmino_last_error", "cimmino_version",
                            "cimmino_opts_default"):
                getattr(L, name).restype = C.c_int
        _lib = L
        return L


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a) -> int:
    return a.data_ptr() if _is_torch(a) else a.ctypes.data


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _check(L, code: int, ctx=None):
    if code != OK:
        msg = L.cimmino_last_error(ctx).decode(errors="replace")
        raise CimminoError(code, msg)


def _opts(L, precision=FP64, layout=SKYLINE, refine_max=None, refine_tol=None,
          pivot_ratio_min=None, max_iter=None, use_graph=None, check_every=None,
          keep_aat=False, refine_relax=None, multi_rhs=None, ruiz_sweeps=None,
          time_proj=None, stream=None, allocator=None, tune=None,
          tune_cache=None) -> OptsStruct:
    o = OptsStruct()
    L.cimmino_opts_default(C.byref(o))
    o.precision = {"fp64": FP64, "fp32_refine": FP32_REFINE}.get(precision, precision)
    o.layout = {"dense": DENSE, "skyline": SKYLINE}.get(layout, layout)
    if refine_max is not None:
        o.refine_max = int(refine_max)
    if refine_tol is not None:
        o.refine_tol = float(refine_tol)
    if pivot_ratio_min is not None:
        o.pivot_ratio_min = float(pivot_ratio_min)
    if max_iter is not None:
        o.max_iter = int(max_iter)
    if use_graph is not None:
        o.use_graph = int(bool(use_graph))
    if check_every is not None:
        o.check_every = int(check_every)
    o.keep_aat = int(bool(keep_aat))
    if multi_rhs is not None:
        # True/1: shared factor reads on CUDA cores; 2: FP32 blocks on the tensor cores
        o.multi_rhs = multi_rhs if isinstance(multi_rhs, int) and not isinstance(
            multi_rhs, bool) else int(bool(multi_rhs))
    if refine_relax is not None:
        o.refine_relax = int(bool(refine_relax))
    if ruiz_sweeps is not None:
        o.ruiz_sweeps = int(ruiz_sweeps)
    if time_proj is not None:
        o.time_proj = int(bool(time_proj))
    o.stream = stream
    if allocator is not None:
        o.alloc, o.free = allocator
    if tune is not None:
        o.tune = int(bool(tune))
    if tune_cache is not None:
        o.tune_cache = os.fsencode(tune_cache)
    return o


def _torch_stream(on_device: bool):
    if not on_device:
        return None
    import torch
    return torch.cuda.current_stream().cuda_stream or None


def _csr(A, keep: list) -> CSRStruct:
    """CSR struct from an object with n, row_ptr, col_idx, val (numpy or torch CUDA)."""
    if _is_torch(A.val):
        dev = True
        arrs = (A.row_ptr, A.col_idx, A.val)
    else:
        dev = False
        arrs = (_host(A.row_ptr, np.int64), _host(A.col_idx, np.int32), _host(A.val, np.float64))
    keep.extend(arrs)
    n = int(A.n)
    return CSRStruct(n, int(arrs[0][-1]) if not dev else int(A.row_ptr[-1].item()),
                     _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]), int(dev))


def _allocator(name):
    if name in (None, "pool"):
        return None
    if name == "torch":
        return torch_allocator()
    raise ValueError(f"allocator must be 'pool' or 'torch', not {name!r}")


class Solver:
    """One system A x = f split into row blocks; FP64 or FP32+refinement factors.

    allocator: "pool" (default) takes device memory from the library's stream-ordered
    pool; "torch" from torch's caching allocator on the context's stream."""

    def __init__(self, A, block_ptr, perm=None, precision="fp64", layout="skyline",
                 allocator=None, **kw):
        L = load()
        self._L = L
        keep: list = []
        csr = _csr(A, keep)
        self.on_device = bool(csr.on_device)
        self.n = int(A.n)
        self.block_ptr = _host(block_ptr, np.int64)
        self.K = len(self.block_ptr) - 1
        self.perm = None if perm is None else _host(perm, np.int32)
        self._alloc = _allocator(allocator)  # kept alive with the context
        opts = _opts(L, precision, layout, stream=_torch_stream(self.on_device),
                     allocator=self._alloc, **kw)
        h = C.c_void_p()
        st = L.cimmino_setup(C.byref(csr), self.K,
                             None if self.perm is None else self.perm.ctypes.data,
                             self.block_ptr.ctypes.data, C.byref(opts), C.byref(h))
        _check(L, st, None)
        self._h = h

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.cimmino_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- solve
    def solve(self, F, tol: float = 1e-10, X=None, raise_on_fail: bool = False):
        """Solve for F of shape (n,) or (nrhs, n) (numpy or torch CUDA).
        Returns (X, [stats dict per right-hand side], status)."""
        L = self._L
        dev = _is_torch(F)
        if dev:
            import torch
            Fm = F.reshape(-1, self.n).contiguous().to(torch.float64)
            if X is None:
                X = torch.empty_like(Fm)
        else:
            Fm = _host(np.atleast_2d(F), np.float64)
            if X is None:
                X = np.empty_like(Fm)
        nrhs = Fm.shape[0]
        stats = (StatsStruct * nrhs)()
        st = L.cimmino_solve(self._h, _ptr(Fm), nrhs, self.n, float(tol), _ptr(X), int(dev), stats)
        # EINVAL / EUNSUPPORTED from a lane (a non-finite right-hand side, or one whose squared
        # norm overflows) comes back with the other lanes' solutions; the same codes from the
        # arguments leave every lane's stats untouched and raise
        lane_einval = st in (EINVAL, EUNSUPPORTED) and any(q.status == st for q in stats)
        if (st not in (OK, ENOCONV, EBREAKDOWN) and not lane_einval) or (raise_on_fail and st != OK):
            _check(L, st, self._h)
        two_d = F.dim() == 2 if dev else np.ndim(F) == 2
        out = X if two_d else X.reshape(self.n)
        return out, [s.as_dict() for s in stats], st

    # -- hooks
    def project(self, v) -> np.ndarray:
        """H v for one n-vector or for each row of an (nrhs, n) array."""
        v = _host(v, np.float64)
        V = np.ascontiguousarray(np.atleast_2d(v))
        out = np.empty_like(V)
        _check(self._L, self._L.cimmino_project(self._h, V.ctypes.data, V.shape[0],
                                                 out.ctypes.data, 0), self._h)
        return out.reshape(v.shape)

    def project_rhs(self, f) -> np.ndarray:
        """xi = sum_i A_i^+ f_i for one n-vector or each row of an (nrhs, n) array."""
        f = _host(f, np.float64)
        Fm = np.ascontiguousarray(np.atleast_2d(f))
        out = np.empty_like(Fm)
        _check(self._L, self._L.cimmino_project_rhs(self._h, Fm.ctypes.data, Fm.shape[0],
                                                     out.ctypes.data, 0), self._h)
        return out.reshape(f.shape)

    def sweeps(self, f, omega: float, sweeps: int) -> np.ndarray:
        """Algorithm 1 from x = 0: `sweeps` block Cimmino sweeps with relaxation omega, for
        one n-vector or each row of an (nrhs, n) array of right-hand sides."""
        f = _host(f, np.float64)
        Fm = np.ascontiguousarray(np.atleast_2d(f))
        out = np.empty_like(Fm)
        _check(self._L, self._L.cimmino_sweeps(self._h, Fm.ctypes.data, Fm.shape[0],
                                                float(omega), int(sweeps), out.ctypes.data, 0),
               self._h)
        return out.reshape(f.shape)

    def aat(self):
        nnz = C.c_int64(0)
        _check(self._L, self._L.cimmino_get_aat_nnz(self._h, C.byref(nnz)), self._h)
        rp = np.empty(self.n + 1, np.int64)
        ci = np.empty(max(nnz.value, 1), np.int32)
        v = np.empty(max(nnz.value, 1), np.float64)
        _check(self._L, self._L.cimmino_get_aat(self._h, rp.ctypes.data, ci.ctypes.data,
                                                 v.ctypes.data), self._h)
        return rp, ci[: nnz.value], v[: nnz.value]

    def colscale(self):
        """Column equilibration divisors cs (ones without equilibration)."""
        cs = np.empty(self.n, np.float64)
        _check(self._L, self._L.cimmino_get_colscale(self._h, cs.ctypes.data), self._h)
        return cs

    def scaled_csr(self, nnz: int):
        """Scaled permuted matrix S (nnz = nnz(A)) and the row factors d, with
        P A = diag(d) S diag(cs)."""
        rp = np.empty(self.n + 1, np.int64)
        ci = np.empty(max(nnz, 1), np.int32)
        v = np.empty(max(nnz, 1), np.float64)
        d = np.empty(self.n, np.float64)
        _check(self._L, self._L.cimmino_get_scaled(self._h, rp.ctypes.data, ci.ctypes.data,
                                                    v.ctypes.data, d.ctypes.data), self._h)
        return rp, ci[:nnz], v[:nnz], d

    def time_kernels(self, reps: int = 10):
        """Average device ms per launch of (projection, A p, A^T y) after a solve."""
        ms = np.zeros(3)
        _check(self._L, self._L.cimmino_time_kernels(self._h, int(reps), ms.ctypes.data), self._h)
        return {"proj_ms": ms[0], "spmv_ms": ms[1], "spmv_t_ms": ms[2]}

    def proj_timing(self):
        """Live projection time of the last solve's CG iterations (opts time_proj=True):
        (summed ms, launches)."""
        ms = C.c_double(0.0)
        n = C.c_int64(0)
        _check(self._L, self._L.cimmino_proj_timing(self._h, C.byref(ms), C.byref(n)), self._h)
        return ms.value, n.value

    def block_rows(self, b: int) -> int:
        m = C.c_int32(0)
        _check(self._L, self._L.cimmino_block_rows(self._h, int(b), C.byref(m)), self._h)
        return m.value

    def factor(self, b: int):
        """Dense copy of L_b (float64) and whether the block was factored in FP64."""
        m = self.block_rows(b)
        Lb = np.empty((m, m), np.float64)
        is64 = C.c_int32(0)
        _check(self._L, self._L.cimmino_get_factor(self._h, int(b), Lb.ctypes.data,
                                                     C.byref(is64)), self._h)
        return Lb, bool(is64.value)


class BatchSolver:
    """Many independent systems solved together (one launch per stage)."""

    def __init__(self, As: Sequence, block_ptrs: Sequence, perms: Optional[Sequence] = None,
                 precision="fp32_refine", layout="skyline", allocator=None, **kw):
        L = load()
        self._L = L
        keep: list = []
        nsys = len(As)
        csrs = (CSRStruct * nsys)(*[_csr(A, keep) for A in As])
        self.ns = [int(A.n) for A in As]
        self._bps = [_host(b, np.int64) for b in block_ptrs]
        Ks = np.asarray([len(b) - 1 for b in self._bps], np.int32)
        bparr = (C.c_void_p * nsys)(*[b.ctypes.data for b in self._bps])
        self._perms = None if perms is None else [None if p is None else _host(p, np.int32)
                                                  for p in perms]
        parr = None if self._perms is None else (C.c_void_p * nsys)(
            *[None if p is None else p.ctypes.data for p in self._perms])
        self._alloc = _allocator(allocator)
        opts = _opts(L, precision, layout, stream=_torch_stream(bool(csrs[0].on_device)),
                     allocator=self._alloc, **kw)
        h = C.c_void_p()
        st = L.cimmino_setup_batch(nsys, csrs, Ks.ctypes.data, parr, bparr, C.byref(opts),
                                   C.byref(h))
        _check(L, st, None)
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.cimmino_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, Fs: Sequence[np.ndarray], tol: float = 1e-10):
        nsys = len(self.ns)
        Fh = [_host(f, np.float64) for f in Fs]
        Xh = [np.empty(n) for n in self.ns]
        farr = (C.c_void_p * nsys)(*[f.ctypes.data for f in Fh])
        xarr = (C.c_void_p * nsys)(*[x.ctypes.data for x in Xh])
        stats = (StatsStruct * nsys)()
        st = self._L.cimmino_solve_batch(self._h, farr, float(tol), xarr, 0, stats)
        lane_einval = st in (EINVAL, EUNSUPPORTED) and any(q.status == st for q in stats)
        if st not in (OK, ENOCONV, EBREAKDOWN) and not lane_einval:
            _check(self._L, st, self._h)
        return Xh, [s.as_dict() for s in stats], st

    def factor(self, q: int, b: int):
        """Dense copy of L of block b of system q, and whether it was factored in FP64."""
        gb = sum(len(bp) - 1 for bp in self._bps[:q]) + int(b)
        m = C.c_int32(0)
        _check(self._L, self._L.cimmino_block_rows(self._h, gb, C.byref(m)), self._h)
        Lb = np.empty((m.value, m.value), np.float64)
        is64 = C.c_int32(0)
        _check(self._L, self._L.cimmino_get_factor(self._h, gb, Lb.ctypes.data, C.byref(is64)),
               self._h)
        return Lb, bool(is64.value)


def aat(A, stream=None):
    """C = A A^T of a host CSR matrix on the GPU (structural pattern, sorted columns)."""
    L = load()
    keep: list = []
    csr = _csr(A, keep)
    nnz = C.c_int64(0)
    rp = np.empty(int(A.n) + 1, np.int64)
    _check(L, L.cimmino_aat(C.byref(csr), stream, C.byref(nnz), rp.ctypes.data, None, None))
    ci = np.empty(max(nnz.value, 1), np.int32)
    v = np.empty(max(nnz.value, 1), np.float64)
    _check(L, L.cimmino_aat(C.byref(csr), stream, C.byref(nnz), rp.ctypes.data, ci.ctypes.data,
                            v.ctypes.data))
    return rp, ci[: nnz.value], v[: nnz.value]


def selftest_wait(limit_us: int = 2000):
    """Watchdog self-test: a device wait on a barrier nothing completes and the FP64
    Cholesky's wait for a partner CTA that never arrives must both give up after limit_us.
    Returns (status code, device error word: 8 | 16); ETIMEOUT is the expected status."""
    L = load()
    word = C.c_int32(0)
    code = L.cimmino_selftest_wait(int(limit_us), C.byref(word))
    return code, word.value


def fp64_peak() -> float:
    """Measured FP64 FMA rate of the current device in TFLOP/s (the FP64 ALU roofline)."""
    L = load()
    t = C.c_double(0.0)
    _check(L, L.cimmino_fp64_peak(C.byref(t)))
    return t.value


def sparsify_dense_columns(A):
    """Copy of A whose dense columns (more than floor(sqrt(n)) nonzeros) keep only their
    floor(sqrt(n)) largest magnitudes (Section 2.3), for building the partitioning graph.
    A has n, row_ptr, col_idx, val (host arrays).  Returns (row_ptr, col_idx, val)."""
    L = load()
    rp, ci, v = _host(A.row_ptr, np.int64), _host(A.col_idx, np.int32), _host(A.val, np.float64)
    n = int(A.n)
    nnz = int(rp[-1])
    orp = np.empty(n + 1, np.int64)
    oci = np.empty(max(nnz, 1), np.int32)
    ov = np.empty(max(nnz, 1), np.float64)
    w = C.c_int64(0)
    _check(L, L.cimmino_sparsify_dense_columns(n, rp.ctypes.data, ci.ctypes.data, v.ctypes.data,
                                               orp.ctypes.data, oci.ctypes.data,
                                               ov.ctypes.data, C.byref(w)))
    return orp, oci[: w.value].copy(), ov[: w.value].copy()


def cholesky_schedule(nt, ntrsm, nfull, maxcta: int, allow_split: bool = True):
    """Static schedule of the FP64 Cholesky for blocks with the given tile counts (host
    only): returns (lists, nsplit, makespan), lists[k] = [(block, part, nparts), ...] of CTA k."""
    L = load()
    nt = _host(nt, np.int32)
    ntrsm, nfull = _host(ntrsm, np.int64), _host(nfull, np.int64)
    nblk = len(nt)
    assert len(ntrsm) == nblk and len(nfull) == nblk
    ncta, nsplit, mk = C.c_int32(0), C.c_int32(0), C.c_double(0.0)
    ptr = np.zeros(int(maxcta) + 1, np.int32)
    items = np.zeros(3 * (nblk + int(maxcta) // 2 + 1), np.int32)
    _check(L, L.cimmino_cholesky_schedule(nblk, nt.ctypes.data, ntrsm.ctypes.data,
                                          nfull.ctypes.data, int(maxcta), int(bool(allow_split)),
                                          C.byref(ncta), ptr.ctypes.data, items.ctypes.data,
                                          C.byref(nsplit), C.byref(mk)))
    it = items.reshape(-1, 3)
    lists = [[tuple(int(v) for v in it[q]) for q in range(ptr[k], ptr[k + 1])]
             for k in range(ncta.value)]
    return lists, int(nsplit.value), float(mk.value)


def partition_rip(n: int, aat_csr, K: int, cap: Optional[int] = None, eps: float = 0.0,
                  seed: int = 0):
    """Graph partition of the row inner-product graph of A (Section 2): aat_csr =
    (row_ptr, col, val) of A A^T for the unscaled A (host arrays, e.g. from ``aat``).  cap
    defaults to ceil(n/K * (1 + eps)).  Returns (perm, block_ptr, cutsize); host only."""
    L = load()
    crp, cci, ccv = (_host(aat_csr[0], np.int64), _host(aat_csr[1], np.int32),
                     _host(aat_csr[2], np.float64))
    if cap is None:
        cap = int(np.ceil(n / K * (1.0 + eps)))
    perm = np.empty(n, np.int32)
    bp = np.empty(K + 1, np.int64)
    cut = C.c_double(0.0)
    _check(L, L.cimmino_partition_rip(int(n), crp.ctypes.data, cci.ctypes.data, ccv.ctypes.data,
                                      int(K), int(cap), int(seed), perm.ctypes.data,
                                      bp.ctypes.data, C.byref(cut)))
    return perm, bp, float(cut.value)

