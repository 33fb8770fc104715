"""Comparison helpers of the GPU parity tests (no method arithmetic)."""
import numpy as np


def rel(a, b):
    """Normwise relative difference ||a - b||_2 / ||b||_2 (Frobenius for matrices)."""
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def assert_close(a, b, tol, what=""):
    """Element by element: every |a_i - b_i| <= tol * max_j |b_j|, so a few wrong small
    entries cannot hide under a norm; the normwise ratio is held to tol as well."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    scale = float(np.abs(b).max()) if b.size else 0.0
    err = np.abs(a - b)
    bad = err > tol * scale
    if bad.any():
        i = np.unravel_index(int(np.argmax(err)), err.shape)
        raise AssertionError(f"{what}: {int(bad.sum())} of {b.size} entries off by more than "
                             f"{tol:g} * max|ref| = {tol * scale:.3e}; worst {err[i]:.3e} at "
                             f"{i} (got {a[i]!r}, expected {b[i]!r})")
    assert rel(a, b) <= tol, (what, rel(a, b))
