"""Failure detection without a GPU fault: a device-side wait that nothing completes gives
up after its budget, the host reads CIMMINO_ETIMEOUT with the device error word, and the
CUDA context stays usable (a solve afterwards still matches the oracle).  Collected last."""
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
    assert code == g.ETIMEOUT and word == 8, (code, word)
    assert dt < 5.0
    w = inputs.workload(1)
    s = g.Solver(w.A, w.block_ptr)
    x, st, code = s.solve(w.F[0], tol=1e-10)
    xo, ito, *_ = oracle.Oracle(w.A, w.block_ptr).solve(w.F[0])
    assert code == 0 and abs(st[0]["iters"] - ito) <= 1
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)

