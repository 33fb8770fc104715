"""Edge cases of the GPU path against the FP64 oracle, through the C ABI: the degenerate
partitions (K = n one-row blocks, K = 1), the largest supported block (4096 rows), a 1 x 1
system, many right-hand sides (three groups of the multi-RHS projection, the last one
partial), and the inputs the setup must reject with a clear error code."""
import numpy as np
import pytest

import inputs
import oracle
from parity_util import assert_close, rel

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_1710_07769_gb300")




@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_refine", 1e-10)])
def test_one_row_blocks(precision, tol):
    """K = n: every G_i is the 1 x 1 block ||r_i||^2 = 1 (after scaling), H = A_s^T A_s
    (Section 1.1 with single-row blocks: the projections onto the rows)."""
    A = inputs.random_dd(300, 4, 21)
    bp = np.arange(A.n + 1, dtype=np.int64)
    s = g.Solver(A, bp, precision=precision)
    o = oracle.Oracle(A, bp)
    v = np.random.default_rng(4).standard_normal(A.n)
    assert_close(s.project(v), o.project(v), tol)
    f = inputs.matvec(A, np.random.default_rng(5).uniform(-1, 1, A.n))
    xo, ito, *_ = o.solve(f)
    x, st, code = s.solve(f)
    assert code == 0 and abs(st[0]["iters"] - ito) <= 1
    assert_close(x, xo, 1e-8)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_refine", 1e-10)])
def test_largest_block(precision, tol):
    """Two blocks of 4096 rows, the largest the projection kernels take (64 tile rows);
    several right-hand sides too (FP64 blocks of this size fall back to one pass per
    right-hand side, FP32 ones to groups of 8)."""
    A = inputs.random_dd(8192, 5, 22)
    bp = np.array([0, 4096, 8192], np.int64)
    s = g.Solver(A, bp, precision=precision)
    o = oracle.Oracle(A, bp, nthreads=2)
    V = np.random.default_rng(6).standard_normal((3, A.n))
    P = s.project(V)
    for k in range(3):
        assert_close(P[k], o.project(V[k]), tol, k)
    for b in (0, 1):
        Lg, is64 = s.factor(b)
        assert_close(np.tril(Lg), o.factor(b), (1e-12 if is64 else 2e-5))


def test_block_over_limit_rejected():
    A = inputs.random_dd(8192, 5, 22)
    with pytest.raises(g.CimminoError) as e:
        g.Solver(A, np.array([0, 4097, 8192], np.int64))
    assert e.value.code == g.EUNSUPPORTED


def test_one_by_one_system():
    """n = 1, K = 1: H = 1, one CG iteration gives x = f / a."""
    A = inputs.CSR(1, np.array([0, 1], np.int64), np.array([0], np.int32), np.array([-4.0]))
    s = g.Solver(A, np.array([0, 1], np.int64))
    x, st, code = s.solve(np.array([2.0]))
    assert code == 0 and st[0]["iters"] == 1
    assert abs(x[0] + 0.5) <= 1e-15


def test_forty_rhs_groups():
    """40 right-hand sides: groups of 16, 16 and 8 (the last one partial) share the factor
    tiles; every column is the oracle's H v."""
    A = inputs.random_dd(700, 5, 11)
    bp = np.array([0, 1, 65, 200, 329, 330, 700], np.int64)
    s = g.Solver(A, bp, precision="fp32_refine")
    o = oracle.Oracle(A, bp)
    V = np.random.default_rng(40).standard_normal((40, A.n))
    P = s.project(V)
    for k in (0, 15, 16, 31, 32, 39):
        assert_close(P[k], o.project(V[k]), 1e-10, k)


def test_bad_inputs_rejected():
    A = inputs.random_dd(200, 4, 3)
    for bp, code in ((np.array([0, 100, 100, 200]), g.EINVAL),   # empty block
                     (np.array([0, 150, 120, 200]), g.EINVAL),   # not increasing
                     (np.array([0, 100, 199]), g.EINVAL),        # does not end at n
                     (np.array([1, 100, 200]), g.EINVAL)):       # does not start at 0
        with pytest.raises(g.CimminoError) as e:
            g.Solver(A, bp.astype(np.int64))
        assert e.value.code == code, bp
    perm = np.arange(200, dtype=np.int32)
    perm[5] = 6  # not a permutation
    with pytest.raises(g.CimminoError) as e:
        g.Solver(A, np.array([0, 100, 200], np.int64), perm=perm)
    assert e.value.code == g.EINVAL
    Z = inputs.CSR(A.n, A.row_ptr.copy(), A.col_idx.copy(), A.val.copy())
    Z.val[Z.row_ptr[7]:Z.row_ptr[8]] = 0.0  # a zero row: A is singular, no unit-norm scaling
    with pytest.raises(g.CimminoError) as e:
        g.Solver(Z, np.array([0, 100, 200], np.int64))
    assert e.value.code == g.ESINGULAR


def test_torch_caching_allocator_callbacks():
    """opts.alloc / opts.free: the context's device memory comes from torch's caching
    allocator (visible in torch's statistics while the context lives, returned on close), and
    the solve equals the one with the library's pool bit for bit."""
    import torch
    w = inputs.workload(1)
    x0, st0, _ = g.Solver(w.A, w.block_ptr, precision="fp32_refine").solve(w.F[0])
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    s = g.Solver(w.A, w.block_ptr, precision="fp32_refine", allocator="torch")
    x1, st1, code = s.solve(w.F[0])
    torch.cuda.synchronize()
    held = torch.cuda.memory_allocated() - before
    assert code == 0 and held >= st1[0]["factor_bytes"]
    s.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    assert st1[0]["iters"] == st0[0]["iters"] and np.array_equal(x1, x0)


def test_projection_autotuner_and_cache(tmp_path):
    """opts.tune: candidate configurations of the projection kernel are timed on the
    context's blocks and the fastest kept; the choice goes to the tuning cache and a second
    context with the same block shape reads it instead of timing.  The arithmetic does not
    depend on the choice, so the solves agree bit for bit with the untuned default."""
    w = inputs.workload(1)
    cache = tmp_path / "tune.txt"
    x0, st0, _ = g.Solver(w.A, w.block_ptr, precision="fp32_refine").solve(w.F[0])
    assert st0[0]["proj_tuned"] == 0 and st0[0]["proj_ctas_per_sm"] == 1
    s1 = g.Solver(w.A, w.block_ptr, precision="fp32_refine", tune=True, tune_cache=str(cache))
    x1, st1, c1 = s1.solve(w.F[0])
    assert c1 == 0 and st1[0]["proj_tuned"] == 1
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and "|fp32|" in lines[0]
    key, minb, slots = lines[0].split()
    assert (int(minb), int(slots)) == (st1[0]["proj_ctas_per_sm"], st1[0]["proj_slots"])
    s2 = g.Solver(w.A, w.block_ptr, precision="fp32_refine", tune=True, tune_cache=str(cache))
    x2, st2, c2 = s2.solve(w.F[0])
    assert st2[0]["proj_tuned"] == 2
    assert (st2[0]["proj_ctas_per_sm"], st2[0]["proj_slots"]) == (int(minb), int(slots))
    assert np.array_equal(x1, x0) and np.array_equal(x2, x0)
    # the two-CTA variant is forced through a cache entry and still agrees bit for bit
    cache.write_text(f"{key} 2 4\n")
    s3 = g.Solver(w.A, w.block_ptr, precision="fp32_refine", tune=True, tune_cache=str(cache))
    x3, st3, _ = s3.solve(w.F[0])
    assert st3[0]["proj_ctas_per_sm"] == 2 and st3[0]["proj_slots"] == 4
    assert np.array_equal(x3, x0)
