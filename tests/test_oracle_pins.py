"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form derived by hand, an independent numpy/LAPACK computation, an invariant
stated in the paper, brute force on tiny inputs, or the one worked number the
paper prints.  None of them retypes the oracle's own formula.
"""
import itertools
import json
import os

import numpy as np
import pytest

import inputs
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense(A):
    return A.to_dense()


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


def small_system(n=96, k=3, seed=7):
    return inputs.random_dd(n, k, seed)


def dense_H(A_scaled_dense, bp):
    """H = sum_i A_i^T (A_i A_i^T)^{-1} A_i with numpy.linalg.solve (independent of the oracle)."""
    n = A_scaled_dense.shape[0]
    H = np.zeros((n, n))
    for b in range(len(bp) - 1):
        Ai = A_scaled_dense[bp[b]:bp[b + 1]]
        H += Ai.T @ np.linalg.solve(Ai @ Ai.T, Ai)
    return H


def oracle_H(o):
    n = o.n
    return np.stack([o.project(np.eye(n)[j]) for j in range(n)], axis=1)


# ---------------------------------------------------------------- SpGEMM (Section 2.3)

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_aat_matches_dense_product(seed):
    A = inputs.random_dd(120, 4, seed)
    crp, cci, cv = oracle.aat_plain(A)
    D = dense(A)
    ref = D @ D.T
    pat = (np.abs(D) > 0).astype(np.int64)
    ref_pat = (pat @ pat.T) > 0                      # structural pattern, integer product
    got = np.zeros_like(ref)
    got_pat = np.zeros(ref.shape, bool)
    for i in range(A.n):
        cols = cci[crp[i]:crp[i + 1]]
        assert np.all(np.diff(cols) > 0), "columns of C must be sorted and unique"
        got[i, cols] = cv[crp[i]:crp[i + 1]]
        got_pat[i, cols] = True
    assert np.array_equal(got_pat, ref_pat)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_aat_keeps_structural_zero():
    # rows 0 and 1 share columns 0 and 1 with products that cancel exactly: 1*1 + 1*(-1) = 0
    D = np.array([[1.0, 1.0, 0.0], [1.0, -1.0, 0.0], [0.0, 0.0, 2.0]])
    crp, cci, cv = oracle.aat_plain(csr_from_dense(D))
    row0 = dict(zip(cci[crp[0]:crp[1]].tolist(), cv[crp[0]:crp[1]].tolist()))
    assert 1 in row0 and row0[1] == 0.0          # kept, value exactly 0.0
    assert 2 not in row0                          # no shared column: no entry


def test_aat_closed_form_2d_stencil_interior():
    """Interior row of C = A A^T for the 5-point upwind stencil (diag a = 4+hb,
    west w = -1-hb, east/north/south -1), derived by hand:
      c_ii = a^2 + w^2 + 3, c_{i,i+-1} = a(w-1), c_{i,i+-2} = -w,
      c_{i,i+-N} = -2a, c_{i,i+-2N} = 1, c_{i,i+-(N+1)} = c_{i,i+-(N-1)} = 1 - w."""
    N, b, h = 16, 20.0, 1.0 / 17
    A = inputs.convdiff2d(N, b, h)
    crp, cci, cv = oracle.aat_plain(A)
    a, w = 4 + h * b, -1 - h * b
    expect = {0: a * a + w * w + 3, 1: a * (w - 1), -1: a * (w - 1), 2: -w, -2: -w,
              N: -2 * a, -N: -2 * a, 2 * N: 1.0, -2 * N: 1.0,
              N + 1: 1 - w, -(N + 1): 1 - w, N - 1: 1 - w, -(N - 1): 1 - w}
    i = 8 * N + 8                                    # far from every boundary
    row = dict(zip(cci[crp[i]:crp[i + 1]].tolist(), cv[crp[i]:crp[i + 1]].tolist()))
    assert sorted(row) == sorted(i + o for o in expect)
    for o, e in expect.items():
        assert row[i + o] == pytest.approx(e, rel=1e-14)


def test_aat_paper_inner_product_216():
    g = json.load(open(os.path.join(GOLDEN, "rip_inner_product_216.json")))
    n = g["n"]
    D = np.zeros((n, n))
    for i in range(n):
        D[i, i] = 1.0 + i          # rows other than r2, r4: a diagonal only
    D[2, :] = 0.0
    D[4, :] = 0.0
    D[2, g["row2"]["cols"]] = g["row2"]["vals"]
    D[4, g["row4"]["cols"]] = g["row4"]["vals"]
    crp, cci, cv = oracle.aat_plain(csr_from_dense(D))
    row = dict(zip(cci[crp[2]:crp[3]].tolist(), cv[crp[2]:crp[3]].tolist()))
    assert row[4] == g["expected_c24"]


def test_scaled_gram_diagonal_is_one():
    """After the Section 2.1 prescaling every row has unit 2-norm, so diag(C) = 1 and
    every |c_ij| is a cosine <= 1 (the edge costs of G_RIP lie in (0, 1])."""
    w = inputs.workload(1)
    o = oracle.Oracle(w.A, w.block_ptr, factor=False)
    crp, cci, cv = o.aat()
    rows = np.repeat(np.arange(o.n), np.diff(crp))
    diag = cv[rows == cci]
    np.testing.assert_allclose(diag, 1.0, rtol=0, atol=4e-16)
    assert np.abs(cv).max() <= 1.0 + 1e-15


# ---------------------------------------------------------------- Cholesky

@pytest.mark.parametrize("m", [1, 2, 7, 33, 64])
def test_cholesky_matches_lapack(m):
    rng = np.random.default_rng(m)
    B = rng.standard_normal((m, m + 3))
    G = B @ B.T
    L, st = oracle.cholesky_dense(G)
    assert st == 0
    np.testing.assert_allclose(L, np.linalg.cholesky(G), rtol=1e-11, atol=1e-12)
    assert np.linalg.norm(L @ L.T - G) / np.linalg.norm(G) < 1e-14


def test_cholesky_detects_non_spd():
    G = np.array([[1.0, 2.0], [2.0, 1.0]])     # eigenvalues 3 and -1
    _, st = oracle.cholesky_dense(G)
    assert st == -2                             # pivot of column 1 is -3 <= 0


def test_block_factor_is_cholesky_of_numpy_gram():
    A = small_system(128, 4, 3)
    bp = np.array([0, 40, 41, 90, 128])         # ragged, with a 1-row block
    o = oracle.Oracle(A, bp)
    rp, ci, v, d = o.scaled()
    S = inputs.CSR(A.n, rp, ci, v).to_dense()
    for b in range(len(bp) - 1):
        Ai = S[bp[b]:bp[b + 1]]
        G = Ai @ Ai.T
        np.testing.assert_allclose(o.gram(b), G, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(o.factor(b), np.linalg.cholesky(G), rtol=1e-11, atol=1e-13)


def test_singular_block_reported():
    D = np.eye(6) * 2.0
    D[1, 4] = 1.0
    D[2] = D[1]                                 # duplicate row -> G_0 singular
    D[2, 2] = 0.0
    D[2, 1] = 2.0
    D[3] = D[1] * 1.0                           # rows 1 and 3 parallel: A_0 rank deficient
    A = csr_from_dense(D)
    with pytest.raises(oracle.OracleError) as e:
        oracle.Oracle(A, np.array([0, 4, 6]))
    assert e.value.code == oracle.ORC_ESINGULAR


# ---------------------------------------------------------------- projections (Eqs. 1.4-1.5, 1.10-1.12)

def test_projection_equals_numpy_pseudoinverse_sum():
    A = small_system(80, 3, 11)
    bp = np.array([0, 17, 50, 80])
    o = oracle.Oracle(A, bp)
    rp, ci, v, d = o.scaled()
    S = inputs.CSR(A.n, rp, ci, v).to_dense()
    H = oracle_H(o)
    Href = dense_H(S, bp)
    np.testing.assert_allclose(H, Href, atol=1e-12)
    # also through the unscaled matrix and numpy's pseudoinverse: H is row-scaling invariant
    D = dense(A)
    Hp = sum(np.linalg.pinv(D[bp[b]:bp[b + 1]]) @ D[bp[b]:bp[b + 1]] for b in range(3))
    np.testing.assert_allclose(H, Hp, atol=1e-11)


def test_projections_symmetric_idempotent_trace():
    A = small_system(72, 4, 5)
    bp = np.array([0, 9, 30, 31, 72])
    o = oracle.Oracle(A, bp)
    H = oracle_H(o)
    assert np.abs(H - H.T).max() < 1e-13
    assert np.trace(H) == pytest.approx(A.n, rel=1e-13)        # sum of ranks m_i
    for b in range(len(bp) - 1):
        ob = oracle.Oracle(A, bp, perm=None)
        # P_b alone: a partition with only block b "active" is emulated by projecting
        # with the block's own rows: P_b = A_b^T G_b^{-1} A_b from the oracle's factor
        L = ob.factor(b)
        rp, ci, v, d = ob.scaled()
        Ab = inputs.CSR(A.n, rp, ci, v).to_dense()[bp[b]:bp[b + 1]]
        Y = np.linalg.solve(L.T, np.linalg.solve(L, Ab))
        P = Ab.T @ Y
        assert np.abs(P @ P - P).max() < 1e-12
        assert np.trace(P) == pytest.approx(bp[b + 1] - bp[b], rel=1e-12)


def test_qr_form_of_H():
    """Eq. 1.10: H = sum_i Q_i Q_i^T with A_i^T = Q_i R_i."""
    A = small_system(60, 3, 21)
    bp = np.array([0, 20, 45, 60])
    H = oracle_H(oracle.Oracle(A, bp))
    D = dense(A)
    Hq = np.zeros_like(H)
    for b in range(3):
        Q, _ = np.linalg.qr(D[bp[b]:bp[b + 1]].T)
        Hq += Q @ Q.T
    np.testing.assert_allclose(H, Hq, atol=1e-12)


def test_K2_spectrum_principal_angles():
    """Eqs. 1.11-1.12 with K = 2: H is similar to [[I, Q1^T Q2], [Q2^T Q1, I]], whose
    eigenvalues are 1 +- sigma_j(Q1^T Q2) plus 1 for the unmatched dimensions."""
    A = small_system(50, 3, 8)
    bp = np.array([0, 22, 50])
    H = oracle_H(oracle.Oracle(A, bp))
    D = dense(A)
    Q1, _ = np.linalg.qr(D[:22].T)
    Q2, _ = np.linalg.qr(D[22:].T)
    s = np.linalg.svd(Q1.T @ Q2, compute_uv=False)
    expect = np.sort(np.concatenate([1 + s, 1 - s, np.ones(50 - 2 * len(s))]))
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(H)), expect, atol=1e-11)


def test_K1_projection_is_identity_and_one_step():
    """K = 1: A_1 = A nonsingular, so H = A^+ A = I and CG converges in one iteration."""
    A = inputs.convdiff2d(24, 20.0)
    n = A.n
    o = oracle.Oracle(A, np.array([0, n]))
    v = np.random.default_rng(0).standard_normal(n)
    np.testing.assert_allclose(o.project(v), v, rtol=0, atol=1e-10 * np.abs(v).max())
    f = inputs.matvec(A, inputs.uniform_x(n, 1, 0)[0])
    x, it, rr, g, st = o.solve(f)
    assert st == 0 and it == 1 and rr <= 1e-10


def test_Kn_is_normal_equations():
    """K = n (one row per block): H = Ahat^T Ahat with Ahat the row-normalised A."""
    A = small_system(40, 3, 2)
    o = oracle.Oracle(A, np.arange(A.n + 1))
    D = dense(A)
    Ah = D / np.linalg.norm(D, axis=1, keepdims=True)
    np.testing.assert_allclose(oracle_H(o), Ah.T @ Ah, atol=1e-13)


def test_row_order_inside_block_irrelevant():
    """Section 2.2: the order of rows inside a block row does not change H."""
    A = small_system(64, 3, 4)
    bp = np.array([0, 20, 64])
    rng = np.random.default_rng(1)
    perm = np.concatenate([rng.permutation(20), 20 + rng.permutation(44)]).astype(np.int32)
    H0 = oracle_H(oracle.Oracle(A, bp))
    H1 = oracle_H(oracle.Oracle(A, bp, perm=perm))
    np.testing.assert_allclose(H0, H1, atol=1e-12)


# ---------------------------------------------------------------- Algorithm 2

def numpy_cg_iterations(H, xi, A, f, tol, maxit=5000):
    """Textbook CG on the dense system (H, xi), stopping on the true residual of A x = f."""
    x = np.zeros_like(xi)
    r = xi.copy()
    p = r.copy()
    rho = r @ r
    nf = np.linalg.norm(f)
    for t in range(maxit):
        q = H @ p
        a = rho / (p @ q)
        x += a * p
        r -= a * q
        rho1 = r @ r
        p = r + (rho1 / rho) * p
        rho = rho1
        if np.linalg.norm(f - A @ x) / nf <= tol:
            return t + 1, x
    return -1, x


@pytest.mark.parametrize("seed,bp", [(3, [0, 30, 70, 100, 150]), (9, [0, 1, 75, 150])])
def test_cg_matches_dense_textbook_cg(seed, bp):
    A = small_system(150, 4, seed)
    bp = np.array(bp)
    D = dense(A)
    xt = np.random.default_rng(seed).uniform(-1, 1, A.n)
    f = D @ xt
    o = oracle.Oracle(A, bp)
    x, it, rr, g, st = o.solve(f)
    rp, ci, v, d = o.scaled()
    S = inputs.CSR(A.n, rp, ci, v).to_dense()
    H = dense_H(S, bp)
    fs = f / np.linalg.norm(D, axis=1)
    xi = S.T @ np.concatenate([np.linalg.solve(S[bp[b]:bp[b + 1]] @ S[bp[b]:bp[b + 1]].T,
                                               fs[bp[b]:bp[b + 1]]) for b in range(len(bp) - 1)])
    it_ref, x_ref = numpy_cg_iterations(H, xi, D, f, 1e-10)
    assert st == 0 and abs(it - it_ref) <= 1
    np.testing.assert_allclose(x, np.linalg.solve(D, f), rtol=0, atol=1e-8)
    # CG bound of Eq. 1.9: after t steps the H-norm error shrinks by 2((sqrt k-1)/(sqrt k+1))^t;
    # the stopping residual 1e-10 is reached well inside the bound for eps = 1e-10 / kappa(A)
    ev = np.linalg.eigvalsh(H)
    kappa = ev[-1] / ev[0]
    assert 0 < ev[0] and ev[-1] <= len(bp) - 1 + 1e-12
    q = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    bound = np.log(1e-10 / (2 * np.linalg.cond(D) * np.sqrt(kappa))) / np.log(q)
    assert it <= np.ceil(bound) + 1


def test_config1_solution_matches_dense_lu():
    w = inputs.workload(1)
    o = oracle.Oracle(w.A, w.block_ptr)
    x, it, rr, g, st = o.solve(w.F[0])
    D = dense(w.A)
    x_lu = np.linalg.solve(D, w.F[0])
    Di = np.linalg.inv(D)
    # kappa_2 <= sqrt(kappa_1 * kappa_inf), cheaper than an SVD of the 4096 x 4096 matrix
    kappa = np.sqrt(np.linalg.norm(D, 1) * np.linalg.norm(D, np.inf)
                    * np.linalg.norm(Di, 1) * np.linalg.norm(Di, np.inf))
    assert st == 0 and rr <= 1e-10 and g < 1e-10
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) <= kappa * 1e-10
    # the spectrum of H lies in (0, K] and its mean is 1 (trace H = n)
    assert 300 < it < 400


def test_gamma_and_first_cg_step_closed_form_2x2():
    """A hand-worked case of Algorithm 2, Eq. 1.5 and Eq. 3.1.  A = [[1, 0], [1, 1]],
    f = (1, 2), one row per block (K = 2).  With unit rows a_1 = (1, 0),
    a_2 = (1, 1)/sqrt(2): H = a_1 a_1^T + a_2 a_2^T = [[3/2, 1/2], [1/2, 1/2]] and
    xi = sum_i A_i^+ f_i = (1, 0) + (1, 1) = (2, 1).  The first CG step from x = 0:
    r = p = xi, rho = 5, p^T H p = (2, 1).(7/2, 3/2) = 17/2, alpha = 10/17, so
    x_1 = (20/17, 10/17) and f - A x_1 = (-3/17, 4/17).  Eq. 3.1 with ||A||_inf = 2,
    ||x_1||_1 = 30/17 and ||f||_inf = 2 gives gamma = (4/17) / (60/17 + 2) = 2/47
    (||x_1||_inf in its place would give 2/37, ||r||_2 would give 5/94); the relative
    2-norm residual is (5/17) / sqrt(5) = sqrt(5)/17."""
    A = inputs.CSR(2, np.array([0, 1, 3], np.int64), np.array([0, 0, 1], np.int32),
                   np.array([1.0, 1.0, 1.0]))
    o = oracle.Oracle(A, np.array([0, 1, 2], np.int64))
    x, it, rr, gam, st = o.solve(np.array([1.0, 2.0]), maxit=1)
    assert it == 1
    np.testing.assert_allclose(x, [20 / 17, 10 / 17], rtol=1e-15)
    assert gam == pytest.approx(2 / 47, rel=1e-14)
    assert rr == pytest.approx(np.sqrt(5) / 17, rel=1e-14)
    # a second step reaches the exact solution x = (1, 1) of the nonsingular 2 x 2 system
    x2, it2, rr2, gam2, st2 = o.solve(np.array([1.0, 2.0]), maxit=2)
    assert st2 == 0 and it2 == 2 and gam2 < 1e-15
    np.testing.assert_allclose(x2, [1.0, 1.0], rtol=1e-14)


@pytest.mark.parametrize("maxit", [3, 40])
def test_gamma_equals_numpy_eq_3_1(maxit):
    """gamma of Eq. 3.1 for the oracle's iterate, recomputed from the dense matrix with
    numpy's norms (infinity norm of A = largest row sum, 1-norm of x)."""
    w = inputs.workload(1)
    o = oracle.Oracle(w.A, w.block_ptr)
    x, it, rr, gam, st = o.solve(w.F[0], maxit=maxit)
    D = dense(w.A)
    f = w.F[0]
    r = D @ x - f
    ref = np.linalg.norm(r, np.inf) / (np.linalg.norm(D, np.inf) * np.linalg.norm(x, 1)
                                       + np.linalg.norm(f, np.inf))
    assert gam == pytest.approx(ref, rel=1e-12)
    assert rr == pytest.approx(np.linalg.norm(r) / np.linalg.norm(f), rel=1e-12)


def test_row_scaling_and_column_permutation_invariance():
    A = small_system(120, 4, 13)
    bp = np.array([0, 40, 80, 120])
    D = dense(A)
    rng = np.random.default_rng(2)
    xt = rng.uniform(-1, 1, A.n)
    f = D @ xt
    x0, it0, *_ = oracle.Oracle(A, bp).solve(f)
    # rows scaled by an arbitrary positive diagonal: same H, same xi (Section 2.1, 3.1)
    s = rng.uniform(0.1, 10, A.n)
    x1, it1, *_ = oracle.Oracle(csr_from_dense(D * s[:, None]), bp).solve(f * s)
    assert abs(it1 - it0) <= 1
    np.testing.assert_allclose(x1, x0, atol=1e-8)
    # columns permuted: the iterates are the permuted iterates (Section 1.2)
    q = rng.permutation(A.n)
    x2, it2, *_ = oracle.Oracle(csr_from_dense(D[:, q]), bp).solve(f)
    assert abs(it2 - it0) <= 1
    np.testing.assert_allclose(x2, x0[q], atol=1e-8)


def test_algorithm1_first_sweep_and_convergence():
    """Algorithm 1 from x^(0) = 0: the first sweep gives omega * xi; with 0 < omega <
    2 / lambda_max(H) the sweeps converge to A^{-1} f."""
    A = small_system(60, 3, 6)
    bp = np.array([0, 20, 40, 60])
    D = dense(A)
    f = D @ np.random.default_rng(3).uniform(-1, 1, A.n)
    o = oracle.Oracle(A, bp)
    np.testing.assert_allclose(o.cimmino_sweeps(f, 0.7, 1), 0.7 * o.project_rhs(f), atol=1e-14)
    lam = np.linalg.eigvalsh(oracle_H(o))
    omega = 2.0 / (lam[0] + lam[-1])
    x = o.cimmino_sweeps(f, omega, 400)
    rate = (lam[-1] - lam[0]) / (lam[-1] + lam[0])
    err = np.linalg.norm(x - np.linalg.solve(D, f)) / np.linalg.norm(np.linalg.solve(D, f))
    assert err <= 10 * np.sqrt(lam[-1] / lam[0]) * rate ** 400 + 1e-12


# ---------------------------------------------------------------- equilibration (Section 3.1)

def badly_scaled(n, seed, spread=3.0):
    """A diagonally dominant sparse matrix with rows and columns multiplied by
    10^U[-spread, spread]: a poorly scaled input (Section 3.1)."""
    D = dense(small_system(n, 4, seed))
    rng = np.random.default_rng(seed + 100)
    D = D * 10.0 ** rng.uniform(-spread, spread, n)[:, None]
    D = D * 10.0 ** rng.uniform(-spread, spread, n)[None, :]
    return csr_from_dense(D), D


def test_equilibration_diagonal_closed_form():
    """A diagonal matrix: the largest entry of row i and column i is |d_i|, so one sweep
    divides by sqrt|d_i| twice and leaves +-1; further sweeps change nothing."""
    rng = np.random.default_rng(31)
    d = rng.choice([-1.0, 1.0], 40) * 10.0 ** rng.uniform(-4, 4, 40)
    A = csr_from_dense(np.diag(d))
    bp = np.arange(0, 41, 8)
    rs, cs = oracle.Oracle(A, bp, ruiz=1).equil()
    np.testing.assert_allclose(rs, np.sqrt(np.abs(d)), rtol=1e-15)
    np.testing.assert_allclose(cs, np.sqrt(np.abs(d)), rtol=1e-15)
    rs5, cs5 = oracle.Oracle(A, bp, ruiz=5).equil()
    np.testing.assert_allclose(rs5 * cs5, np.abs(d), rtol=4e-16 * 8)
    o = oracle.Oracle(A, bp, ruiz=5)
    x, it, rr, g, st = o.solve(d * np.arange(1, 41))
    assert st == 0 and it == 1      # Ae = sign(D): every block projection is exact
    np.testing.assert_allclose(x, np.arange(1, 41), rtol=1e-14)


def test_equilibration_rank_one_closed_form():
    """A = u v^T (positive): row max u_i max(v), column max max(u) v_j, so one sweep
    gives rs_i = sqrt(u_i max v), cs_j = sqrt(max u v_j) and
    Ae_ij = sqrt(u_i v_j / (max u max v)).  One-row blocks keep every G_i nonsingular."""
    rng = np.random.default_rng(32)
    u, v = rng.uniform(0.1, 100, 9), rng.uniform(0.1, 100, 9)
    A = csr_from_dense(np.outer(u, v))
    o = oracle.Oracle(A, np.arange(10), ruiz=1)
    rs, cs = o.equil()
    np.testing.assert_allclose(rs, np.sqrt(u * v.max()), rtol=2e-16 * 4)
    np.testing.assert_allclose(cs, np.sqrt(u.max() * v), rtol=2e-16 * 4)
    Ae = np.outer(u, v) / np.outer(rs, cs)
    np.testing.assert_allclose(Ae, np.sqrt(np.outer(u, v) / (u.max() * v.max())), rtol=1e-15)


def test_equilibration_converges_and_factors_reconstruct_A():
    """After k sweeps every row and column of Ae has largest magnitude close to one
    (Section 3.1), and A = diag(d) S diag(cs) for the scaled permuted rows S."""
    A, D = badly_scaled(150, 33, spread=4.0)
    bp = np.array([0, 50, 100, 150])
    perm = np.random.default_rng(5).permutation(150).astype(np.int32)
    o = oracle.Oracle(A, bp, perm=perm, factor=False, ruiz=30)
    rs, cs = o.equil()
    Ae = D / np.outer(rs, cs)
    dev = max(np.abs(np.abs(Ae).max(axis=1) - 1).max(), np.abs(np.abs(Ae).max(axis=0) - 1).max())
    assert dev <= 1e-6, dev
    rp, ci, v, d = o.scaled()
    S = inputs.CSR(150, rp, ci, v).to_dense()
    np.testing.assert_allclose(d[:, None] * S * cs[None, :], D[perm], rtol=1e-13)
    assert np.allclose(np.linalg.norm(S, axis=1), 1.0, rtol=1e-15)


def test_equilibrated_projection_is_column_scaled_pseudoinverse_sum():
    """Column scaling changes H (Section 3.1): with equilibration the oracle's H is
    sum_i pinv(B_i) B_i for B = A diag(1/cs), not the H of A."""
    A, D = badly_scaled(60, 34)
    bp = np.array([0, 20, 45, 60])
    o = oracle.Oracle(A, bp, ruiz=8)
    rs, cs = o.equil()
    B = D / cs[None, :]
    Href = sum(np.linalg.pinv(B[bp[b]:bp[b + 1]]) @ B[bp[b]:bp[b + 1]] for b in range(3))
    H = oracle_H(o)
    np.testing.assert_allclose(H, Href, atol=1e-10)
    H0 = oracle_H(oracle.Oracle(A, bp))
    assert np.abs(H - H0).max() > 0.1
    assert np.trace(H) == pytest.approx(60, rel=1e-12)   # still a sum of projections


def test_equilibrated_solve_matches_dense_lu_and_preconditions():
    """With equilibration the solve still reaches A^{-1} f, K = 1 still takes one step,
    and on a badly column-scaled matrix it takes fewer CG iterations than without
    (column scaling acts as a preconditioner, Section 3.1).  Algorithm 1 returns x too."""
    A, D = badly_scaled(120, 35)
    bp = np.array([0, 30, 60, 90, 120])
    xt = np.random.default_rng(9).uniform(-1, 1, 120)
    f = D @ xt
    x_lu = np.linalg.solve(D, f)
    kappa = np.linalg.cond(D)
    x1, it1, rr1, g1, st1 = oracle.Oracle(A, bp, ruiz=10).solve(f)
    x0, it0, rr0, g0, st0 = oracle.Oracle(A, bp).solve(f)
    assert st1 == 0 and rr1 <= 1e-10
    assert np.linalg.norm(x1 - x_lu) <= kappa * 1e-10 * np.linalg.norm(x_lu)
    assert st0 == 0 and it1 < it0, (it1, it0)
    xk, itk, *_ = oracle.Oracle(A, np.array([0, 120]), ruiz=10).solve(f)
    assert itk == 1 and np.linalg.norm(xk - x_lu) <= kappa * 1e-14 * np.linalg.norm(x_lu)
    # Algorithm 1 on the equilibrated system: the first sweep is omega * xi in the
    # column-scaled space, returned as x = y / cs; the sweeps converge to A^{-1} f
    A, D = badly_scaled(60, 36, spread=1.0)
    bp = np.array([0, 20, 40, 60])
    f = D @ xt[:60]
    o = oracle.Oracle(A, bp, ruiz=10)
    cs = o.equil()[1]
    np.testing.assert_allclose(o.cimmino_sweeps(f, 0.7, 1) * cs, 0.7 * o.project_rhs(f),
                               rtol=1e-14, atol=1e-300)
    lam = np.linalg.eigvalsh(oracle_H(o))
    xs = o.cimmino_sweeps(f, 2.0 / (lam[0] + lam[-1]), 400)
    rate = (lam[-1] - lam[0]) / (lam[-1] + lam[0])
    bound = 10 * np.sqrt(lam[-1] / lam[0]) * rate ** 400 * cs.max() / cs.min()
    assert bound < 1e-4
    x_lu = np.linalg.solve(D, f)
    assert np.linalg.norm(xs - x_lu) / np.linalg.norm(x_lu) <= bound + 1e-12


def test_zero_rhs_and_zero_row():
    w = inputs.workload(1)
    o = oracle.Oracle(w.A, w.block_ptr)
    x, it, rr, g, st = o.solve(np.zeros(w.A.n))
    assert st == 0 and it == 0 and not x.any()
    D = np.eye(4)
    D[2, 2] = 0.0
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(csr_from_dense(D + np.diag([0, 0, 0, 0])), np.array([0, 2, 4]))


# ---------------------------------------------------------------- partition metrics (Eqs. 2.6-2.9)

def test_cutsize_equals_interblock_sum_and_ip_matrix():
    A = small_system(90, 4, 17)
    crp, cci, cv = oracle.aat_plain(A)
    D = dense(A)
    C = D @ D.T
    part = np.random.default_rng(0).integers(0, 4, A.n).astype(np.int32)
    cut = oracle.cutsize(crp, cci, cv, part)
    mask = part[:, None] != part[None, :]
    assert cut == pytest.approx(np.abs(C[mask]).sum() / 2, rel=1e-12)
    ip = oracle.ip_matrix(crp, cci, cv, part, 4)
    for k in range(4):
        for m in range(4):
            if k != m:
                blk = np.abs(C[np.ix_(part == k, part == m)]).sum()
                assert ip[k, m] == pytest.approx(blk, rel=1e-12)
    off = ip.sum() - np.trace(ip)
    assert off == pytest.approx(2 * cut, rel=1e-12)


def test_cutsize_brute_force_bisection():
    """Every balanced 2-way partition of a 10-row matrix: the oracle's cutsize equals the
    sum of |r_i r_j^T| over pairs split by the partition computed by brute force."""
    A = inputs.random_dd(10, 2, 4)
    D = dense(A)
    crp, cci, cv = oracle.aat_plain(A)
    best = None
    for left in itertools.combinations(range(10), 5):
        part = np.ones(10, np.int32)
        part[list(left)] = 0
        brute = sum(abs(D[i] @ D[j]) for i in range(10) for j in range(i + 1, 10)
                    if part[i] != part[j])
        cut = oracle.cutsize(crp, cci, cv, part)
        assert cut == pytest.approx(brute, rel=1e-12, abs=1e-12)
        best = cut if best is None else min(best, cut)
    assert best >= 0


# ---------------------------------------------------------------- dense columns (Section 2.3)

def numpy_sparsify(D):
    """Independent restatement on a dense array: keep the floor(sqrt(n)) largest
    magnitudes of every column with more nonzeros than that (lower row first on ties)."""
    n = D.shape[0]
    t = int(np.floor(np.sqrt(n)))
    out = D.copy()
    for j in range(n):
        rows = np.nonzero(D[:, j])[0]
        if len(rows) > t:
            order = np.lexsort((rows, -np.abs(D[rows, j])))
            out[rows[order[t:]], j] = 0.0
    return out


def test_dense_column_example_25():
    """The paper's example: n = 25 and one column with 23 nonzeros; sqrt(25) = 5, so the
    column keeps its 5 largest entries and the other columns are untouched."""
    ex = json.load(open(os.path.join(GOLDEN, "dense_column_25.json")))
    n = ex["n"]
    rng = np.random.default_rng(12)
    D = np.diag(rng.uniform(1, 2, n))
    rows = np.sort(rng.choice(n, ex["dense_column_nnz"], replace=False))
    D[rows, 3] = rng.uniform(-5, 5, len(rows))
    D[3, 3] = 9.0
    A = csr_from_dense(D)
    assert np.count_nonzero(D[:, 3]) == ex["dense_column_nnz"]
    rp, ci, v = oracle.sparsify_dense_columns(A)
    S = inputs.CSR(n, rp, ci, v).to_dense()
    assert np.count_nonzero(S[:, 3]) == ex["kept"]
    kept = np.sort(np.abs(S[:, 3][S[:, 3] != 0]))
    assert np.array_equal(kept, np.sort(np.abs(D[:, 3]))[-ex["kept"]:])
    others = [j for j in range(n) if j != 3]
    assert np.array_equal(S[:, others], D[:, others])


@pytest.mark.parametrize("n,seed", [(50, 1), (144, 2), (200, 3)])
def test_dense_columns_match_numpy_and_sparsify_graph(n, seed):
    """Several dense columns with tied magnitudes: the same entries as an independent
    numpy restatement; C of the sparsified matrix has fewer nonzeros; a matrix without
    dense columns comes back unchanged."""
    rng = np.random.default_rng(seed)
    D = np.diag(rng.uniform(1, 2, n)) + np.diag(-np.ones(n - 1), 1)
    for j in rng.choice(n, 3, replace=False):
        rows = rng.choice(n, n // 2, replace=False)
        D[rows, j] = rng.choice([-2.0, -1.0, 1.0, 3.0], len(rows))   # many ties
    A = csr_from_dense(D)
    rp, ci, v = oracle.sparsify_dense_columns(A)
    S = inputs.CSR(n, rp, ci, v).to_dense()
    assert np.array_equal(S, numpy_sparsify(D))
    assert len(oracle.aat_plain(inputs.CSR(n, rp, ci, v))[1]) < len(oracle.aat_plain(A)[1])
    # the boundary: a column with floor(sqrt(n)) + 1 nonzeros is dense, one with
    # floor(sqrt(n)) is not
    t = int(np.floor(np.sqrt(n)))
    E = np.diag(rng.uniform(1, 2, n))
    E[rng.choice(np.arange(1, n), t, replace=False), 0] = rng.uniform(3, 4, t)      # t + 1
    E[rng.choice(np.arange(0, n - 1), t - 1, replace=False), n - 1] = 5.0           # t
    rp3, ci3, v3 = oracle.sparsify_dense_columns(csr_from_dense(E))
    S3 = inputs.CSR(n, rp3, ci3, v3).to_dense()
    assert np.count_nonzero(S3[:, 0]) == t and np.count_nonzero(E[:, 0]) == t + 1
    assert np.array_equal(S3[:, 1:], E[:, 1:])
    B = inputs.convdiff2d(12, 20.0)
    rp2, ci2, v2 = oracle.sparsify_dense_columns(B)
    assert np.array_equal(rp2, B.row_ptr) and np.array_equal(ci2, B.col_idx)
    assert np.array_equal(v2, B.val)


def test_range_factor_and_solves_equal_full_setup():
    """The bounded-sample entry points (Cholesky and inner solves of a range of blocks)
    reproduce numpy's solves with the Gram blocks of the full setup, and touch only their
    own blocks' rows."""
    A = inputs.random_dd(700, 5, 11)
    bp = np.array([0, 1, 65, 200, 329, 330, 700], np.int64)
    perm = np.random.default_rng(5).permutation(700).astype(np.int32)
    full = oracle.Oracle(A, bp, perm=perm)
    part = oracle.Oracle(A, bp, perm=perm, factor=False)
    assert part.factor_range(2, 5) == 0
    u = np.random.default_rng(3).standard_normal(700)
    y = part.solve_range(u)
    for b in (2, 3, 4):
        r0, r1 = bp[b], bp[b + 1]
        np.testing.assert_allclose(y[r0:r1], np.linalg.solve(full.gram(b), u[r0:r1]),
                                   rtol=1e-11, atol=1e-13)
    assert not y[:bp[2]].any() and not y[bp[5]:].any()
