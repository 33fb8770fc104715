"""GPU path against the FP64 oracle, element by element, through the C ABI.

Tolerances (stated requirements of the method's implementation):
  * pattern of C = A A^T: bit-exact; values of C: 1e-12 relative;
  * FP64 factors L_i: 1e-12 relative (Frobenius) against the oracle's L_i;
  * FP64 projections H v: 1e-12 relative (2-norm);
  * solves: relative residual <= 1e-10 and the oracle's iteration count +-1;
  * FP32+refinement: inner solves refined to ||G y - u|| <= 1e-12 ||u||, so each y_i
    is within kappa(G_i) * 1e-12 of the exact solve; with kappa(G_i) < 100 for the
    test blocks, H v agrees to 1e-10 relative, and the iteration count to +-1.
Sizes span several 64-row tiles with ragged tails and 1-row blocks.
"""
import numpy as np
import pytest

import inputs
import oracle
from parity_util import assert_close, rel

pytestmark = pytest.mark.gpu

g = pytest.importorskip("paper_1710_07769_gb300")




def csr_from_dense(D):
    n = D.shape[0]
    rp = np.zeros(n + 1, np.int64)
    cols, vals = [], []
    for i in range(n):
        nz = np.nonzero(D[i])[0]
        cols.append(nz)
        vals.append(D[i, nz])
        rp[i + 1] = rp[i] + len(nz)
    return inputs.CSR(n, rp, np.concatenate(cols).astype(np.int32), np.concatenate(vals))


RAGGED = np.array([0, 1, 65, 200, 329, 330, 700], np.int64)  # m = 1, 64, 135, 129, 1, 370


@pytest.fixture(scope="module")
def sys_small():
    A = inputs.random_dd(700, 5, 11)
    rng = np.random.default_rng(5)
    perm = rng.permutation(700).astype(np.int32)
    xt = rng.uniform(-1, 1, 700)
    return A, perm, inputs.matvec(A, xt)


# ------------------------------------------------------------------ SpGEMM (Section 2.3)

@pytest.mark.parametrize("which", ["random", "stencil2d", "stencil3d"])
def test_aat_standalone_bitexact(which):
    A = {"random": lambda: inputs.random_dd(3000, 8, 3),
         "stencil2d": lambda: inputs.convdiff2d(40, 20.0),
         "stencil3d": lambda: inputs.convdiff3d(12, 11, 10, (30, 20, 10))}[which]()
    rp, ci, v = g.aat(A)
    orp, oci, ov = oracle.aat_plain(A)
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci)      # pattern bit-exact
    np.testing.assert_allclose(v, ov, rtol=1e-12, atol=0)
    assert np.array_equal(v, ov)                                   # same sum order: bitwise


def test_aat_dense_column_overflow_path():
    """A column with 1500 entries gives rows with more than 1024 candidates (CTA path)."""
    n = 2000
    D = np.zeros((n, n))
    D[np.arange(n), np.arange(n)] = 3.0
    D[:1500, 7] += np.linspace(0.5, 1.5, 1500)
    A = csr_from_dense(D)
    rp, ci, v = g.aat(A)
    orp, oci, ov = oracle.aat_plain(A)
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci)
    np.testing.assert_allclose(v, ov, rtol=1e-12)


def test_setup_scaled_and_aat_match_oracle(sys_small):
    A, perm, f = sys_small
    s = g.Solver(A, RAGGED, perm=perm, keep_aat=True)
    o = oracle.Oracle(A, RAGGED, perm=perm)
    rp, ci, v, d = s.scaled_csr(A.nnz)
    orp, oci, ov, od = o.scaled()
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci)
    np.testing.assert_allclose(v, ov, rtol=1e-15, atol=0)
    np.testing.assert_allclose(d, od, rtol=1e-15)
    crp, cci, cv = s.aat()
    ocrp, occi, ocv = o.aat()
    assert np.array_equal(crp, ocrp) and np.array_equal(cci, occi)
    np.testing.assert_allclose(cv, ocv, rtol=1e-12, atol=1e-15)


def _dense_column_system():
    """2000 rows, a column with 1500 entries: rows with more than 1024 candidates."""
    n = 2000
    D = np.zeros((n, n))
    D[np.arange(n), np.arange(n)] = 3.0
    D[:1500, 7] += np.linspace(0.5, 1.5, 1500)
    D[np.arange(1, n), np.arange(n - 1)] -= 0.4
    return csr_from_dense(D), np.array([0, 700, 1400, 2000], np.int64)


@pytest.mark.parametrize("case", ["ragged", "dense_column"])
def test_gram_blocks_direct_equal_cut_from_full_c(sys_small, case):
    """Without opts.keep_aat the setup forms the Gram blocks G_i directly: each row of
    C = A A^T gathers only the candidates of its own block (Section 2.3 restricted to the
    block diagonal).  The blocks, hence the factors and H v, are bit for bit those cut from
    the full C; the dense column sends rows through the CTA path of the SpGEMM."""
    if case == "ragged":
        A, perm, f = sys_small
        bp = RAGGED
    else:
        A, bp = _dense_column_system()
        perm = None
    s_full = g.Solver(A, bp, perm=perm, keep_aat=True, precision="fp64")
    s_direct = g.Solver(A, bp, perm=perm, precision="fp64")
    for b in range(len(bp) - 1):
        assert np.array_equal(s_full.factor(b)[0], s_direct.factor(b)[0]), b
    v = np.random.default_rng(41).standard_normal(A.n)
    assert np.array_equal(s_full.project(v), s_direct.project(v))
    x1, st1, c1 = s_full.solve(inputs.matvec(A, v))
    x2, st2, c2 = s_direct.solve(inputs.matvec(A, v))
    assert c1 == c2 == 0 and st2[0]["nnz_aat"] == 0 and st1[0]["nnz_aat"] > st2[0]["nnz_gram"]
    assert st1[0]["nnz_gram"] == st2[0]["nnz_gram"]
    assert np.array_equal(x1, x2)
    s_full.close()
    s_direct.close()


# ------------------------------------------------------------------ Cholesky of G_i

@pytest.mark.parametrize("layout", ["dense", "skyline"])
def test_fp64_factors_match_oracle(sys_small, layout):
    A, perm, f = sys_small
    s = g.Solver(A, RAGGED, perm=perm, layout=layout)
    o = oracle.Oracle(A, RAGGED, perm=perm)
    for b in range(len(RAGGED) - 1):
        Lg, is64 = s.factor(b)
        assert is64
        assert_close(Lg, o.factor(b), 1e-12, b)


def test_fp64_factors_stencil_skyline_envelope():
    """Contiguous blocks of a 3D stencil: G_i is banded, the skyline layout stores only
    the envelope, and the factor still equals the oracle's dense Cholesky factor."""
    A = inputs.convdiff3d(16, 16, 6, (30, 20, 10))
    bp = inputs.contiguous_blocks(A.n, 700)
    s = g.Solver(A, bp, layout="skyline")
    o = oracle.Oracle(A, bp)
    for b in [0, len(bp) - 2]:
        Lg, _ = s.factor(b)
        assert_close(Lg, o.factor(b), 1e-12)


def test_fp64_split_block_matches_oracle():
    """A block that would set the FP64 Cholesky's time on its own (2048 rows with a dense
    envelope, beside 40 one-tile blocks) is shared by two CTAs that meet at pair barriers:
    its factor, the small blocks' factors, the projection (Eq. 1.5) and the solve still
    equal the oracle's."""
    A = inputs.random_dd(2048 + 40 * 64, 8, 31)
    bp = np.concatenate([[0], 2048 + 64 * np.arange(41)]).astype(np.int64)
    s = g.Solver(A, bp)
    o = oracle.Oracle(A, bp, nthreads=2)
    f = inputs.matvec(A, np.random.default_rng(4).uniform(-1, 1, A.n))
    x, st, code = s.solve(f, tol=1e-10)
    assert code == 0 and st[0]["chol_split_blocks"] >= 1, st[0]
    for b in (0, 1, 40):
        Lg, is64 = s.factor(b)
        assert is64
        assert_close(Lg, o.factor(b), 1e-12, b)
    v = np.random.default_rng(2).standard_normal(A.n)
    assert_close(s.project(v), o.project(v), 1e-12)
    xo, ito, *_ = o.solve(f)
    assert abs(st[0]["iters"] - ito) <= 1
    assert_close(x, xo, 1e-8)


def test_fp32_factors_close_to_oracle(sys_small):
    A, perm, f = sys_small
    s = g.Solver(A, RAGGED, perm=perm, precision="fp32_refine")
    o = oracle.Oracle(A, RAGGED, perm=perm)
    for b in range(len(RAGGED) - 1):
        Lg, is64 = s.factor(b)
        tol = 1e-12 if is64 else 2e-5
        assert_close(Lg, o.factor(b), tol, b)


# ------------------------------------------------------------------ projections (Eq. 1.5)

@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_refine", 1e-10)])
def test_projection_matches_oracle(sys_small, precision, tol):
    A, perm, f = sys_small
    s = g.Solver(A, RAGGED, perm=perm, precision=precision)
    o = oracle.Oracle(A, RAGGED, perm=perm)
    v = np.random.default_rng(1).standard_normal(A.n)
    assert_close(s.project(v), o.project(v), tol)
    assert_close(s.project_rhs(f), o.project_rhs(f), tol)


# ------------------------------------------------------------------ Algorithm 2

@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("layout", ["dense", "skyline"])
def test_config1_solve_matches_oracle(precision, layout):
    w = inputs.workload(1)
    o = oracle.Oracle(w.A, w.block_ptr)
    xo, ito, rro, go, sto = o.solve(w.F[0])
    s = g.Solver(w.A, w.block_ptr, precision=precision, layout=layout)
    x, st, code = s.solve(w.F[0], tol=1e-10)
    assert code == 0 and st[0]["status"] == 0
    assert abs(st[0]["iters"] - ito) <= 1, (st[0]["iters"], ito)
    assert st[0]["rel_res"] <= 1e-10
    r = np.linalg.norm(w.F[0] - inputs.matvec(w.A, x)) / np.linalg.norm(w.F[0])
    assert r <= 1.01e-10
    # both solutions are within kappa * 1e-10 of the truth; kappa(A) of config 1 is < 50
    assert_close(x, xo, 1e-8)


def test_solve_ragged_permuted_matches_oracle(sys_small):
    A, perm, f = sys_small
    o = oracle.Oracle(A, RAGGED, perm=perm)
    xo, ito, *_ = o.solve(f)
    for precision in ("fp64", "fp32_refine"):
        s = g.Solver(A, RAGGED, perm=perm, precision=precision)
        x, st, code = s.solve(f)
        assert code == 0 and abs(st[0]["iters"] - ito) <= 1
        assert_close(x, xo, 1e-8)


def test_K1_one_iteration():
    A = inputs.convdiff2d(50, 20.0)
    f = inputs.matvec(A, inputs.uniform_x(A.n, 1, 3)[0])
    s = g.Solver(A, np.array([0, A.n]))
    x, st, code = s.solve(f)
    assert code == 0 and st[0]["iters"] == 1


def test_zero_rhs_gives_zero():
    w = inputs.workload(1)
    s = g.Solver(w.A, w.block_ptr)
    x, st, code = s.solve(np.zeros(w.A.n))
    assert code == 0 and st[0]["iters"] == 0 and not np.any(x)


def test_multi_rhs_matches_single(sys_small):
    A, perm, f = sys_small
    rng = np.random.default_rng(9)
    F = np.stack([inputs.matvec(A, rng.uniform(-1, 1, A.n)) for _ in range(3)])
    o = oracle.Oracle(A, RAGGED, perm=perm)
    s = g.Solver(A, RAGGED, perm=perm, precision="fp32_refine")
    X, st, code = s.solve(F)
    assert code == 0
    for k in range(3):
        xo, ito, *_ = o.solve(F[k])
        assert abs(st[k]["iters"] - ito) <= 1
        assert_close(X[k], xo, 1e-8)


def test_deterministic_bitwise():
    w = inputs.workload(1)
    s = g.Solver(w.A, w.block_ptr, precision="fp32_refine")
    x1, s1, _ = s.solve(w.F[0])
    x2, s2, _ = s.solve(w.F[0])
    assert np.array_equal(x1, x2) and s1[0]["iters"] == s2[0]["iters"]


def test_graph_and_eager_agree():
    w = inputs.workload(1)
    x1, s1, _ = g.Solver(w.A, w.block_ptr, use_graph=True, check_every=5).solve(w.F[0])
    x2, s2, _ = g.Solver(w.A, w.block_ptr, use_graph=False, check_every=1).solve(w.F[0])
    assert s1[0]["iters"] == s2[0]["iters"]
    assert np.array_equal(x1, x2)


def test_batch_matches_individual_oracles():
    systems = inputs.batch_workload(nsys=4, seed=4, max_nz=6)
    bs = g.BatchSolver([w.A for w in systems], [w.block_ptr for w in systems])
    X, st, code = bs.solve([w.F[0] for w in systems])
    assert code == 0
    for w, x, s in zip(systems, X, st):
        xo, ito, *_ = oracle.Oracle(w.A, w.block_ptr).solve(w.F[0])
        assert abs(s["iters"] - ito) <= 1
        assert_close(x, xo, 1e-8)


# ------------------------------------------------------------------ errors

def test_errors_reported():
    w = inputs.workload(1)
    bad = inputs.CSR(w.A.n, w.A.row_ptr.copy(), w.A.col_idx.copy(), w.A.val)
    bad.col_idx[5] = w.A.n + 3
    with pytest.raises(g.CimminoError) as e:
        g.Solver(bad, w.block_ptr)
    assert e.value.code == g.EINVAL
    # rank-deficient block: two parallel rows in block 0
    D = np.eye(8) * 2.0
    D[1] = D[0] * 3.0
    with pytest.raises(g.CimminoError) as e:
        g.Solver(csr_from_dense(D), np.array([0, 4, 8]))
    assert e.value.code == g.ESINGULAR
    s = g.Solver(w.A, w.block_ptr, max_iter=3)
    x, st, code = s.solve(w.F[0])
    assert code == g.ENOCONV and st[0]["iters"] == 3


# ------------------------------------------------------------------ several right-hand sides

def envelope_matrix():
    """640 rows, 2 blocks of 320 (5 tiles each): tridiagonal A gives a pentadiagonal G_i
    with tile envelope J0 = [0, 0, 1, 2, .]; one long-range entry in row 261 (tile 4)
    reaching column 74 couples tile 4 with tile 1, so J0(4) = 1 < J0(3) = 2 (a
    non-monotone envelope: the backward chain of tile row 1 meets a zero tile at J = 3)."""
    n = 640
    D = np.zeros((n, n))
    i = np.arange(n)
    D[i, i] = 4.0
    D[i[1:], i[:-1]] = -1.3
    D[i[:-1], i[1:]] = -0.7
    D[261, 74] = 0.9
    D[320 + 261, 320 + 74] = -0.6
    return csr_from_dense(D), np.array([0, 320, 640], np.int64)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_refine", 1e-10)])
@pytest.mark.parametrize("nrhs", [2, 8, 11, 16, 21])
def test_projection_multi_rhs_matches_oracle(sys_small, precision, tol, nrhs):
    """Groups of 8 or 16 right-hand sides share each factor tile (padded and partial
    groups included); every column equals the oracle's H v."""
    A, perm, f = sys_small
    s = g.Solver(A, RAGGED, perm=perm, precision=precision)
    o = oracle.Oracle(A, RAGGED, perm=perm)
    V = np.random.default_rng(nrhs).standard_normal((nrhs, A.n))
    P = s.project(V)
    for k in range(nrhs):
        assert_close(P[k], o.project(V[k]), tol, k)
    Fm = np.stack([inputs.matvec(A, V[k]) for k in range(nrhs)])
    Xi = s.project_rhs(Fm)
    for k in range(0, nrhs, 5):
        assert_close(Xi[k], o.project_rhs(Fm[k]), tol, k)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_refine", 1e-10)])
def test_projection_multi_rhs_nonmonotone_envelope(precision, tol):
    A, bp = envelope_matrix()
    o = oracle.Oracle(A, bp)
    V = np.random.default_rng(3).standard_normal((16, A.n))
    for multi in (2, True, False):  # tensor cores (FP32 blocks), CUDA cores, one per RHS
        s = g.Solver(A, bp, precision=precision, multi_rhs=multi)
        P = s.project(V)
        for k in range(16):
            assert_close(P[k], o.project(V[k]), tol, (multi, k))


@pytest.mark.parametrize("nrhs", [3, 16, 21])
def test_multi_rhs_tensor_cores_and_cuda_cores_match_oracle(sys_small, nrhs):
    """Algorithm 2 step 5 for several right-hand sides sharing the FP32 factors: on the
    tensor cores (multi_rhs = 2: 3xTF32 MMAs, W in tensor memory) and on CUDA cores
    (multi_rhs = 1), each column element by element against the oracle's H v (Eq. 1.5);
    the solve reports every block on the tensor-core kernel in the first case only."""
    A, perm, f = sys_small
    o = oracle.Oracle(A, RAGGED, perm=perm)
    V = np.random.default_rng(100 + nrhs).standard_normal((nrhs, A.n))
    F = np.stack([inputs.matvec(A, V[k]) for k in range(nrhs)])
    ref = [o.project(V[k]) for k in range(nrhs)]
    for mode, ntc in ((2, len(RAGGED) - 1), (1, 0)):
        s = g.Solver(A, RAGGED, perm=perm, precision="fp32_refine", multi_rhs=mode)
        P = s.project(V)
        for k in range(nrhs):
            assert_close(P[k], ref[k], 1e-10, (mode, k))
        X, st, code = s.solve(F)
        assert code == 0 and all(q["mr_tc_blocks"] == ntc for q in st), (mode, st[0])
        for k in (0, nrhs - 1):
            assert_close(X[k], V[k], 1e-8, (mode, k))
        s.close()


def test_multi_rhs_large_block_takes_cuda_cores():
    """A block of 33 tile rows (2060 rows) is beyond the tensor-core kernel's 32; it runs
    on the CUDA-core kernel in the same projection as the tensor-core blocks."""
    A = inputs.random_dd(2600, 4, 17)
    bp = np.array([0, 2060, 2071, 2600], np.int64)
    o = oracle.Oracle(A, bp)
    V = np.random.default_rng(31).standard_normal((16, A.n))
    s = g.Solver(A, bp, precision="fp32_refine", multi_rhs=2)
    P = s.project(V)
    for k in (0, 7, 15):
        assert_close(P[k], o.project(V[k]), 1e-10, k)
    F = np.stack([inputs.matvec(A, V[k]) for k in range(16)])
    X, st, code = s.solve(F)
    assert code == 0 and st[0]["mr_tc_blocks"] == 2
    assert_close(X[5], V[5], 1e-8)


def test_solve_16_rhs_matches_oracle():
    """16 independent CG lanes sharing the factors (the multi-right-hand-side reading):
    each lane's iteration count and solution against its own oracle solve."""
    w = inputs.workload(1)
    rng = np.random.default_rng(21)
    F = np.stack([inputs.matvec(w.A, rng.uniform(-1, 1, w.A.n)) for _ in range(16)])
    s = g.Solver(w.A, w.block_ptr, precision="fp32_refine")
    X, st, code = s.solve(F)
    assert code == 0
    o = oracle.Oracle(w.A, w.block_ptr)
    for k in range(16):
        xo, ito, *_ = o.solve(F[k])
        assert st[k]["status"] == 0 and abs(st[k]["iters"] - ito) <= 1, (k, st[k]["iters"], ito)
        assert st[k]["rel_res"] <= 1e-10
        assert_close(X[k], xo, 1e-8)
    # the same lanes through one factor pass per right-hand side, and with the triangular
    # solves of the 16 lanes on the tensor cores
    for multi in (False, 2):
        X2, st2, _ = g.Solver(w.A, w.block_ptr, precision="fp32_refine",
                              multi_rhs=multi).solve(F)
        for k in range(16):
            assert abs(st2[k]["iters"] - st[k]["iters"]) <= 1, (multi, k)
            assert_close(X2[k], X[k], 1e-8, (multi, k))


# ------------------------------------------------------------------ relaxed inner tolerance

def test_relaxed_inner_tolerance_converges():
    """refine_relax: inner solves to refine_tol / relres_t (capped at 1e-6) inside CG
    iterations.  Same stopping test (true residual <= 1e-10); fewer refinement steps than
    exact inner solves; against the oracle's exact-projection CG (Algorithm 2): the
    iteration count within 1% (+1) and x within 1e-8 element by element."""
    w = inputs.workload(1)
    xo, ito, *_ = oracle.Oracle(w.A, w.block_ptr).solve(w.F[0])
    ex = g.Solver(w.A, w.block_ptr, precision="fp32_refine")
    x0, s0, c0 = ex.solve(w.F[0])
    rx = g.Solver(w.A, w.block_ptr, precision="fp32_refine", refine_relax=True)
    x1, s1, c1 = rx.solve(w.F[0])
    assert c0 == 0 and c1 == 0
    assert s1[0]["rel_res"] <= 1e-10
    r = np.linalg.norm(w.F[0] - inputs.matvec(w.A, x1)) / np.linalg.norm(w.F[0])
    assert r <= 1.01e-10
    assert s1[0]["refine_steps_total"] < s0[0]["refine_steps_total"]
    assert abs(s1[0]["iters"] - ito) <= 1 + ito // 100, (s1[0]["iters"], ito)
    assert_close(x1, xo, 1e-8)


# ------------------------------------------------------------------ FP64 refactorisation

# Per-block min_j L_jj^2 of the oracle's FP64 factors of sys_small with RAGGED blocks:
# 1.0, 0.846, 0.776, 0.737, 1.0, 0.634.  A pivot-ratio threshold of 0.8 therefore sends
# exactly blocks 2, 3 and 5 to the FP64 refactorisation (FP32 pivots differ from these by
# ~1e-6, far from the threshold), leaving 0, 1 and 4 in FP32: a mixed context.
FALLBACK_BLOCKS = {2, 3, 5}


def test_fp64_fallback_mixed_context(sys_small):
    A, perm, f = sys_small
    o = oracle.Oracle(A, RAGGED, perm=perm)
    for b in range(len(RAGGED) - 1):  # the premise of the threshold, from the oracle
        piv = float((np.diag(o.factor(b)) ** 2).min())
        assert (piv < 0.8) == (b in FALLBACK_BLOCKS), (b, piv)
    s = g.Solver(A, RAGGED, perm=perm, precision="fp32_refine", pivot_ratio_min=0.8)
    for b in range(len(RAGGED) - 1):
        Lg, is64 = s.factor(b)
        assert is64 == (b in FALLBACK_BLOCKS), b
        assert_close(Lg, o.factor(b), 1e-12 if is64 else 2e-5, b)
    # H v and xi through the mixed FP32 / FP64 projection (single and several vectors)
    v = np.random.default_rng(12).standard_normal(A.n)
    assert_close(s.project(v), o.project(v), 1e-10, "H v")
    assert_close(s.project_rhs(f), o.project_rhs(f), 1e-10, "xi")
    V = np.random.default_rng(13).standard_normal((11, A.n))
    P = s.project(V)
    for k in range(11):
        assert_close(P[k], o.project(V[k]), 1e-10, k)
    # FP32 blocks on the tensor-core kernel, the FP64 ones on the CUDA-core kernel
    s2 = g.Solver(A, RAGGED, perm=perm, precision="fp32_refine", pivot_ratio_min=0.8,
                  multi_rhs=2)
    P2 = s2.project(V)
    for k in range(11):
        assert_close(P2[k], o.project(V[k]), 1e-10, ("tc", k))
    s2.close()
    xo, ito, *_ = o.solve(f)
    x, st, code = s.solve(f)
    assert code == 0 and st[0]["fallbacks"] == len(FALLBACK_BLOCKS)
    assert abs(st[0]["iters"] - ito) <= 1, (st[0]["iters"], ito)
    assert_close(x, xo, 1e-8)


# ------------------------------------------------------------------ graph partition (Section 2)

def _gp_case(which):
    if which == "stencil":  # the 64^3 workload's generator at 16^3, K = 8, eps = 5%
        w = inputs.workload(2, scale="small")
        return w.A, w.F[0], len(w.block_ptr) - 1, int(np.floor(1.05 * w.A.n / (len(w.block_ptr) - 1)))
    A = inputs.random_dd(700, 5, 11)
    f = inputs.matvec(A, np.random.default_rng(6).uniform(-1, 1, A.n))
    return A, f, 6, 130


@pytest.mark.parametrize("which", ["stencil", "random"])
def test_graph_partition_solve_matches_oracle(which):
    """Blocks from the host partitioner of the row inner-product graph (uneven sizes, RCM
    order inside blocks, wide skylines): the partition is an input to both sides, and the
    GPU solve must match the oracle's Algorithm 2 on it."""
    A, f, K, cap = _gp_case(which)
    perm, bp, cut = g.partition_rip(A.n, g.aat(A), K, cap=cap, seed=0)
    sizes = np.diff(bp)
    assert sizes.max() <= cap and sizes.min() >= 1 and len(np.unique(sizes)) > 1
    assert sorted(perm.tolist()) == list(range(A.n))
    o = oracle.Oracle(A, bp, perm=perm)
    xo, ito, *_ = o.solve(f)
    v = np.random.default_rng(4).standard_normal(A.n)
    for precision, tol in (("fp64", 1e-12), ("fp32_refine", 1e-10)):
        s = g.Solver(A, bp, perm=perm, precision=precision)
        assert_close(s.project(v), o.project(v), tol, precision)
        x, st, code = s.solve(f)
        assert code == 0 and abs(st[0]["iters"] - ito) <= 1, (precision, st[0]["iters"], ito)
        assert_close(x, xo, 1e-8, precision)
        s.close()


# ------------------------------------------------------------------ Algorithm 1

@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32_refine", 1e-9)])
def test_cimmino_sweeps_match_oracle(sys_small, precision, tol):
    """Algorithm 1 from x = 0 on the same setup: the first sweep is omega * xi, later
    sweeps follow the oracle's iterates; two right-hand sides at once."""
    A, perm, f = sys_small
    s = g.Solver(A, RAGGED, perm=perm, precision=precision)
    o = oracle.Oracle(A, RAGGED, perm=perm)
    x1 = s.sweeps(f, 0.7, 1)
    assert_close(x1, 0.7 * o.project_rhs(f), tol)
    F = np.stack([f, inputs.matvec(A, np.random.default_rng(2).uniform(-1, 1, A.n))])
    for sweeps in (5, 30):
        X = s.sweeps(F, 1.3, sweeps)
        for k in range(2):
            assert_close(X[k], o.cimmino_sweeps(F[k], 1.3, sweeps), tol, (sweeps, k))


# ------------------------------------------------------------------ equilibration (Section 3.1)

@pytest.fixture(scope="module")
def sys_badly_scaled():
    """The 700-row random matrix with rows and columns multiplied by 10^U[-1.5,1.5]: the
    oracle's CG takes 3596 iterations without equilibration and 125-128 with 10 sweeps.
    (With a wider spread the residual creeps across 1e-10 by a few percent per
    iteration, and rounding alone moves the crossing by more than one iteration.)"""
    A = inputs.random_dd(700, 5, 11)
    rng = np.random.default_rng(41)
    rf, cf = 10.0 ** rng.uniform(-1.5, 1.5, 700), 10.0 ** rng.uniform(-1.5, 1.5, 700)
    rows = np.repeat(np.arange(700), np.diff(A.row_ptr))
    B = inputs.CSR(700, A.row_ptr.copy(), A.col_idx.copy(), A.val * rf[rows] * cf[A.col_idx])
    perm = np.random.default_rng(5).permutation(700).astype(np.int32)
    F = np.stack([inputs.matvec(B, rng.uniform(-1, 1, 700)) for _ in range(3)])
    return B, perm, F, oracle.Oracle(B, RAGGED, perm=perm, ruiz=10)


def kappa2(B):
    return np.linalg.cond(B.to_dense())


def test_equilibration_setup_bitwise(sys_badly_scaled):
    """Equilibrated, row-normalised, permuted matrix, its row factors d and the column
    divisors cs: the same rounded operations in the same order on both sides."""
    B, perm, F, o = sys_badly_scaled
    s = g.Solver(B, RAGGED, perm=perm, ruiz_sweeps=10)
    rp, ci, v, d = s.scaled_csr(B.nnz)
    orp, oci, ov, od = o.scaled()
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci)
    assert np.array_equal(v, ov) and np.array_equal(d, od)
    assert np.array_equal(s.colscale(), o.equil()[1])
    assert np.array_equal(g.Solver(B, RAGGED, perm=perm).colscale(), np.ones(700))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_refine", 1e-10)])
def test_equilibrated_projection_and_solve_match_oracle(sys_badly_scaled, precision, tol):
    """H of the column-scaled system (FP32 blocks: kappa(G_i) <= 72, so the refined inner
    solves hold H v to 1e-10); three right-hand sides solved at
    once, each returned as x = y / cs, with the oracle's iteration count +-1 and gamma."""
    B, perm, F, o = sys_badly_scaled
    s = g.Solver(B, RAGGED, perm=perm, precision=precision, ruiz_sweeps=10)
    v = np.random.default_rng(8).standard_normal(700)
    assert_close(s.project(v), o.project(v), tol)
    assert_close(s.project_rhs(F[0]), o.project_rhs(F[0]), tol)
    X, st, code = s.solve(F)
    assert code == 0
    # two x with relative residual <= 1e-10 differ by at most 2 kappa(A) 1e-10 relative
    # (kappa(A) is about 1.2e6 here); a wrong column unscaling is off by O(1)
    xbound = 2 * kappa2(B) * 1e-10
    for k in range(3):
        xo, ito, rro, go, sto = o.solve(F[k])
        assert sto == 0 and abs(st[k]["iters"] - ito) <= 1, (k, st[k]["iters"], ito)
        assert st[k]["rel_res"] <= 1e-10
        assert_close(X[k], xo, xbound, k)
        # gamma of Eq. 3.1 for the returned x, recomputed on the host with the original A
        res = F[k] - inputs.matvec(B, X[k])
        ainf = np.add.reduceat(np.abs(B.val), B.row_ptr[:-1]).max()
        gam = np.abs(res).max() / (ainf * np.abs(X[k]).sum() + np.abs(F[k]).max())
        assert st[k]["backward_err"] == pytest.approx(gam, rel=0.05)
    # one right-hand side alone (the single-vector kernels) reaches the same x
    x1, st1, code1 = s.solve(F[1])
    assert code1 == 0 and abs(st1[0]["iters"] - st[1]["iters"]) <= 1
    assert_close(x1, o.solve(F[1])[0], xbound)


def test_equilibrated_sweeps_match_oracle(sys_badly_scaled):
    B, perm, F, o = sys_badly_scaled
    s = g.Solver(B, RAGGED, perm=perm, ruiz_sweeps=10)
    for sweeps in (1, 12):
        X = s.sweeps(F[:2], 0.9, sweeps)
        for k in range(2):
            assert_close(X[k], o.cimmino_sweeps(F[k], 0.9, sweeps), 1e-11, (sweeps, k))


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_live_projection_timing(sys_small, precision):
    """opts time_proj records CUDA events around every projection launch of the CG loop
    (eager launches): the same iterates bit for bit as the graph-launched solve, and one
    timed launch per iteration that produced the returned x."""
    A, perm, f = sys_small
    ref = g.Solver(A, RAGGED, perm=perm, precision=precision)
    x0, st0, _ = ref.solve(f)
    for use_graph in (True, False):
        s = g.Solver(A, RAGGED, perm=perm, precision=precision, time_proj=True,
                     use_graph=use_graph)
        x, st, code = s.solve(f)
        assert code == 0 and st[0]["iters"] == st0[0]["iters"]
        assert np.array_equal(x, x0)
        ms, n = s.proj_timing()
        assert n == st[0]["iters"] and ms > 0.0
        s.close()
    with pytest.raises(g.CimminoError):
        ref.proj_timing()
