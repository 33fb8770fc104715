"""Failure detection without a GPU fault: device-side waits that nothing completes (the
projection ring's mbarrier wait, bit 8; the FP64 Cholesky's wait for the other CTA of a split
block, bit 16) give up after their budget, the host reads CIMMINO_ETIMEOUT with the device
error word, and the
CUDA context stays usable (a solve afterwards still matches the oracle); a non-finite
right-hand side is reported as an input error, and one whose squared norm overflows FP64 as
beyond the solver's range."""
import time

import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_1710_07769_gb300")


def test_bounded_wait_reports_timeout_and_context_survives():
    t0 = time.perf_counter()
    code, word = g.selftest_wait(limit_us=2000)
    dt = time.perf_counter() - t0
    assert code == g.ETIMEOUT and word == 8 | 16, (code, word)
    assert dt < 5.0
    w = inputs.workload(1)
    s = g.Solver(w.A, w.block_ptr)
    x, st, code = s.solve(w.F[0], tol=1e-10)
    xo, ito, *_ = oracle.Oracle(w.A, w.block_ptr).solve(w.F[0])
    assert code == 0 and abs(st[0]["iters"] - ito) <= 1
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)



def test_nonfinite_rhs_is_an_input_error():
    """A right-hand side holding NaN (or Inf) stops its lane with EINVAL instead of being
    taken for a zero vector; the other lanes of the same solve are unaffected."""
    w = inputs.workload(1)
    s = g.Solver(w.A, w.block_ptr)
    F = np.stack([w.F[0], w.F[0].copy(), w.F[0]])
    F[1, 17] = np.nan
    X, st, code = s.solve(F, tol=1e-10)
    assert code == g.EINVAL
    assert st[1]["status"] == g.EINVAL and not X[1].any()
    for k in (0, 2):
        assert st[k]["status"] == 0 and st[k]["rel_res"] <= 1e-10


def test_overflowing_rhs_norm_is_reported_as_such():
    """Finite entries of 1e160 overflow ||f||^2 in FP64: that lane stops with EUNSUPPORTED and
    a message naming the overflow (not NaN / Inf), while the other lanes still converge."""
    w = inputs.workload(1)
    s = g.Solver(w.A, w.block_ptr)
    F = np.stack([w.F[0], 1e160 * w.F[0], w.F[0]])
    X, st, code = s.solve(F, tol=1e-10)
    assert code == g.EUNSUPPORTED
    assert st[1]["status"] == g.EUNSUPPORTED and not X[1].any()
    msg = s._L.cimmino_last_error(s._h).decode()
    assert "overflows" in msg and "NaN" not in msg, msg
    for k in (0, 2):
        assert st[k]["status"] == 0 and st[k]["rel_res"] <= 1e-10
