/*
 * Plain FP64 CPU oracle for the CG-accelerated block Cimmino solve
 * (Torun, Manguoglu, Aykanat, "A Novel Partitioning Method for Accelerating
 * the Block Cimmino Algorithm", arXiv 1710.07769).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it and shares no code,
 * header, table or helper with it.
 *
 * Everything is written as the plain definition in plain loops, in double
 * precision, compiled without floating-point contraction:
 *   - optional row and column infinity-norm equilibration before the row
 *     2-norm step (Section 3.1: the iterative procedure that brings the largest
 *     entry of every row and column to one; column scaling changes H and acts
 *     as a preconditioner, row scaling does not);
 *   - row 2-norm prescaling (Section 2.1) and the row permutation A^Pi = P A
 *     decoded from a partition (Section 2.2);
 *   - C = A A^T by row-wise Gustavson SpGEMM (Section 2.3, "Constructing
 *     G_RIP"); the pattern is structural (entries that cancel to 0.0 stay);
 *   - the Gram blocks G_i = A_i A_i^T (the diagonal blocks of C) and their
 *     Cholesky factors, used to apply A_i^+ = A_i^T (A_i A_i^T)^{-1}
 *     (Section 1, pseudoinverse definition) without forming it;
 *   - the projection sum H v = sum_i A_i^+ A_i v (Eq. 1.5);
 *   - Algorithm 2 (classical CG on H x = xi, xi = sum_i A_i^+ f_i,
 *     Section 1.1) with x^(0) = 0 (Section 3.1), stopping on the true
 *     relative residual ||f - A x||_2 / ||f||_2 and also reporting the
 *     normwise backward error gamma of Eq. 3.1;
 *   - Algorithm 1 (block Cimmino with relaxation omega);
 *   - the dense-column rule for building the graph (Section 2.3): a column with
 *     more than sqrt(n) nonzeros keeps only its sqrt(n) largest magnitudes;
 *   - the partition metrics cutsize(Pi) = interIP(Pi) (Eqs. 2.6-2.7) and the
 *     inter-block inner-product matrix ip_km (Eqs. 2.8-2.9).
 *
 * Threads: OpenMP (when enabled) only splits independent blocks or
 * independent columns; every sum keeps the same order as the sequential
 * program, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ESINGULAR (-3)
#define ORC_ENOCONV (-4)
#define ORC_EBREAKDOWN (-5)

typedef struct orc_ctx {
  int64_t n, nnz;
  int32_t K;
  /* factors of a sub-range of blocks [rb0, rb1) only (bounded CPU timing samples) */
  int32_t rb0, rb1;
  int64_t *rfoff;
  double *rL;
  /* original matrix (for the true residual) */
  int64_t *rp0;
  int32_t *ci0;
  double *v0;
  /* scaled, permuted matrix A^Pi = D^{-1} P A (CSR) */
  int64_t *rp;
  int32_t *ci;
  double *v;
  double *d;     /* original row perm[r] = d[r] * (scaled row r) * diag(cs) */
  /* equilibration (Section 3.1): A = diag(rs) Ae diag(cs); all ones when off */
  int32_t ruiz;  /* equilibration sweeps (0 = off) */
  double *rs, *cs;
  double *ve;    /* values of Ae (pattern of the original matrix) */
  int32_t *perm; /* permuted row r is original row perm[r] */
  int64_t *bp;   /* block r-ranges over permuted rows, K+1 */
  /* column-wise copy of the scaled permuted matrix (CSC), rows increasing */
  int64_t *cp;
  int32_t *ri;
  double *cv;
  /* C = A A^T of the scaled permuted matrix (CSR, columns increasing) */
  int64_t *crp;
  int32_t *cci;
  double *ccv;
  int64_t nnzc;
  /* Cholesky factors, one packed lower triangle (row-major) per block */
  int64_t *foff;
  double *L;
  int32_t fail_block;
  int nthreads;
} orc_ctx;

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

/* ---- Section 3.1: row and column infinity-norm equilibration ----
 * One sweep takes, on the current matrix Ae, the largest magnitude of every row
 * (rmax_i) and of every column (cmax_j), and divides entry (i, j) by
 * sqrt(rmax_i) * sqrt(cmax_j); rs_i and cs_j accumulate the divisors, so that
 * A = diag(rs) Ae diag(cs) holds throughout.  An empty row or column keeps the
 * divisor 1.  The largest entry of every row and column tends to one. */
static int equilibrate(orc_ctx *c) {
  int64_t n = c->n;
  c->rs = (double *)xcalloc(n, sizeof(double));
  c->cs = (double *)xcalloc(n, sizeof(double));
  c->ve = (double *)xcalloc(c->nnz, sizeof(double));
  double *rmax = (double *)xcalloc(n, sizeof(double));
  double *cmax = (double *)xcalloc(n, sizeof(double));
  if (!c->rs || !c->cs || !c->ve || !rmax || !cmax) { free(rmax); free(cmax); return ORC_ENOMEM; }
  for (int64_t i = 0; i < n; ++i) c->rs[i] = c->cs[i] = 1.0;
  memcpy(c->ve, c->v0, sizeof(double) * (size_t)c->nnz);
  for (int32_t sweep = 0; sweep < c->ruiz; ++sweep) {
    for (int64_t i = 0; i < n; ++i) rmax[i] = cmax[i] = 0.0;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t q = c->rp0[i]; q < c->rp0[i + 1]; ++q) {
        double a = fabs(c->ve[q]);
        if (a > rmax[i]) rmax[i] = a;
        if (a > cmax[c->ci0[q]]) cmax[c->ci0[q]] = a;
      }
    for (int64_t i = 0; i < n; ++i) {
      rmax[i] = rmax[i] > 0.0 ? sqrt(rmax[i]) : 1.0;
      cmax[i] = cmax[i] > 0.0 ? sqrt(cmax[i]) : 1.0;
    }
    for (int64_t i = 0; i < n; ++i)
      for (int64_t q = c->rp0[i]; q < c->rp0[i + 1]; ++q)
        c->ve[q] = c->ve[q] / (rmax[i] * cmax[c->ci0[q]]);
    for (int64_t i = 0; i < n; ++i) {
      c->rs[i] = c->rs[i] * rmax[i];
      c->cs[i] = c->cs[i] * cmax[i];
    }
  }
  free(rmax);
  free(cmax);
  return ORC_OK;
}

/* ---- Section 2.1: scale every row to unit 2-norm; Section 2.2: permute rows ----
 * The input is the equilibrated matrix Ae (the original one when equilibration
 * is off); d[r] carries both row factors back to the original row. */
static int scale_permute(orc_ctx *c) {
  int64_t n = c->n;
  c->rp = (int64_t *)xcalloc(n + 1, sizeof(int64_t));
  c->ci = (int32_t *)xcalloc(c->nnz, sizeof(int32_t));
  c->v = (double *)xcalloc(c->nnz, sizeof(double));
  c->d = (double *)xcalloc(n, sizeof(double));
  if (!c->rp || !c->ci || !c->v || !c->d) return ORC_ENOMEM;
  c->rp[0] = 0;
  for (int64_t r = 0; r < n; ++r) {
    int64_t o = c->perm[r];
    c->rp[r + 1] = c->rp[r] + (c->rp0[o + 1] - c->rp0[o]);
  }
  for (int64_t r = 0; r < n; ++r) {
    int64_t o = c->perm[r];
    double ss = 0.0;
    for (int64_t q = c->rp0[o]; q < c->rp0[o + 1]; ++q) ss += c->ve[q] * c->ve[q];
    double nr = sqrt(ss);
    if (!(nr > 0.0)) return ORC_ESINGULAR; /* an empty / zero row makes A singular */
    c->d[r] = c->ruiz > 0 ? nr * c->rs[o] : nr;
    int64_t w = c->rp[r];
    for (int64_t q = c->rp0[o]; q < c->rp0[o + 1]; ++q, ++w) {
      c->ci[w] = c->ci0[q];
      c->v[w] = c->ve[q] / nr;
    }
  }
  return ORC_OK;
}

/* column-wise (CSC) copy: stable counting sort, rows increasing inside a column */
static int transpose(orc_ctx *c) {
  int64_t n = c->n;
  c->cp = (int64_t *)xcalloc(n + 1, sizeof(int64_t));
  c->ri = (int32_t *)xcalloc(c->nnz, sizeof(int32_t));
  c->cv = (double *)xcalloc(c->nnz, sizeof(double));
  int64_t *fill = (int64_t *)xcalloc(n, sizeof(int64_t));
  if (!c->cp || !c->ri || !c->cv || !fill) { free(fill); return ORC_ENOMEM; }
  for (int64_t q = 0; q < c->nnz; ++q) c->cp[c->ci[q] + 1]++;
  for (int64_t k = 0; k < n; ++k) c->cp[k + 1] += c->cp[k];
  for (int64_t k = 0; k < n; ++k) fill[k] = c->cp[k];
  for (int64_t r = 0; r < n; ++r)
    for (int64_t q = c->rp[r]; q < c->rp[r + 1]; ++q) {
      int64_t w = fill[c->ci[q]]++;
      c->ri[w] = (int32_t)r;
      c->cv[w] = c->v[q];
    }
  free(fill);
  return ORC_OK;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* ---- Section 2.3: C = A A^T by Gustavson's row-wise SpGEMM ----
 * row i of C: for every a_ik of row i (k increasing) and every a_jk of
 * column k (j increasing), c_ij += a_ik * a_jk.  An entry exists as soon as
 * rows i and j share a column (structural pattern), whatever its value. */
static int aat(orc_ctx *c) {
  int64_t n = c->n;
  int32_t *mark = (int32_t *)xcalloc(n, sizeof(int32_t));
  double *acc = (double *)xcalloc(n, sizeof(double));
  int32_t *list = (int32_t *)xcalloc(n, sizeof(int32_t));
  c->crp = (int64_t *)xcalloc(n + 1, sizeof(int64_t));
  if (!mark || !acc || !list || !c->crp) { free(mark); free(acc); free(list); return ORC_ENOMEM; }
  for (int64_t j = 0; j < n; ++j) mark[j] = -1;
  /* symbolic pass: count distinct j per row */
  for (int64_t i = 0; i < n; ++i) {
    int64_t cnt = 0;
    for (int64_t q = c->rp[i]; q < c->rp[i + 1]; ++q) {
      int32_t k = c->ci[q];
      for (int64_t s = c->cp[k]; s < c->cp[k + 1]; ++s) {
        int32_t j = c->ri[s];
        if (mark[j] != (int32_t)i) { mark[j] = (int32_t)i; ++cnt; }
      }
    }
    c->crp[i + 1] = c->crp[i] + cnt;
  }
  c->nnzc = c->crp[n];
  c->cci = (int32_t *)xcalloc(c->nnzc, sizeof(int32_t));
  c->ccv = (double *)xcalloc(c->nnzc, sizeof(double));
  if (!c->cci || !c->ccv) { free(mark); free(acc); free(list); return ORC_ENOMEM; }
  for (int64_t j = 0; j < n; ++j) mark[j] = -1;
  /* numeric pass */
  for (int64_t i = 0; i < n; ++i) {
    int64_t cnt = 0;
    for (int64_t q = c->rp[i]; q < c->rp[i + 1]; ++q) {
      int32_t k = c->ci[q];
      double aik = c->v[q];
      for (int64_t s = c->cp[k]; s < c->cp[k + 1]; ++s) {
        int32_t j = c->ri[s];
        double prod = aik * c->cv[s];
        if (mark[j] != (int32_t)i) {
          mark[j] = (int32_t)i;
          acc[j] = prod;
          list[cnt++] = j;
        } else {
          acc[j] = acc[j] + prod;
        }
      }
    }
    qsort(list, (size_t)cnt, sizeof(int32_t), cmp_i32);
    int64_t w = c->crp[i];
    for (int64_t t = 0; t < cnt; ++t, ++w) {
      c->cci[w] = list[t];
      c->ccv[w] = acc[list[t]];
    }
  }
  free(mark); free(acc); free(list);
  return ORC_OK;
}

/* ---- Cholesky G = L L^T of one dense SPD block (row-oriented, plain definition) ----
 * L is packed lower row-major: L(i,j) at i*(i+1)/2 + j.  Returns 0, or
 * -(j+1) when the pivot of column j is not positive (G not SPD, i.e. the
 * block A_i is rank deficient). */
static int64_t pk(int64_t i, int64_t j) { return i * (i + 1) / 2 + j; }

static int cholesky_packed(int64_t m, double *L) {
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t j = 0; j <= i; ++j) {
      double s = L[pk(i, j)];
      for (int64_t k = 0; k < j; ++k) s -= L[pk(i, k)] * L[pk(j, k)];
      if (i == j) {
        if (!(s > 0.0)) return (int)(-(j + 1));
        L[pk(i, i)] = sqrt(s);
      } else {
        L[pk(i, j)] = s / L[pk(j, j)];
      }
    }
  }
  return 0;
}

/* G_i = C restricted to the rows and columns of block i (lower triangle) */
static void gram_block(const orc_ctx *c, int32_t b, double *G) {
  int64_t r0 = c->bp[b], r1 = c->bp[b + 1];
  int64_t m = r1 - r0;
  memset(G, 0, sizeof(double) * (size_t)(m * (m + 1) / 2));
  for (int64_t i = r0; i < r1; ++i)
    for (int64_t q = c->crp[i]; q < c->crp[i + 1]; ++q) {
      int64_t j = c->cci[q];
      if (j >= r0 && j <= i) G[pk(i - r0, j - r0)] = c->ccv[q];
    }
}

static int factor_all(orc_ctx *c) {
  int32_t K = c->K;
  c->foff = (int64_t *)xcalloc((size_t)K + 1, sizeof(int64_t));
  if (!c->foff) return ORC_ENOMEM;
  for (int32_t b = 0; b < K; ++b) {
    int64_t m = c->bp[b + 1] - c->bp[b];
    c->foff[b + 1] = c->foff[b] + m * (m + 1) / 2;
  }
  c->L = (double *)xcalloc((size_t)c->foff[K], sizeof(double));
  if (!c->L) return ORC_ENOMEM;
  int fail = -1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(c->nthreads)
  for (int32_t b = 0; b < K; ++b) {
    int64_t m = c->bp[b + 1] - c->bp[b];
    double *L = c->L + c->foff[b];
    gram_block(c, b, L);
    if (cholesky_packed(m, L) != 0) {
#pragma omp critical
      { if (fail < 0 || b < fail) fail = b; }
    }
  }
  c->fail_block = fail;
  return fail >= 0 ? ORC_ESINGULAR : ORC_OK;
}

/* forward solve L z = b, then backward solve L^T y = z (in place in y) */
static void chol_solve(int64_t m, const double *L, const double *b, double *y) {
  for (int64_t i = 0; i < m; ++i) {
    double s = b[i];
    for (int64_t k = 0; k < i; ++k) s -= L[pk(i, k)] * y[k];
    y[i] = s / L[pk(i, i)];
  }
  for (int64_t i = m - 1; i >= 0; --i) {
    double s = y[i];
    for (int64_t k = i + 1; k < m; ++k) s -= L[pk(k, i)] * y[k];
    y[i] = s / L[pk(i, i)];
  }
}

/* y_i = G_i^{-1} u_i for every block; u and y are permuted-row vectors */
static void block_solves(const orc_ctx *c, const double *u, double *y) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(c->nthreads)
  for (int32_t b = 0; b < c->K; ++b) {
    int64_t r0 = c->bp[b], m = c->bp[b + 1] - r0;
    chol_solve(m, c->L + c->foff[b], u + r0, y + r0);
  }
}

/* u = A^Pi v  (rows of the scaled permuted matrix, k increasing) */
static void spmv(const orc_ctx *c, const double *v, double *u) {
#pragma omp parallel for schedule(static) num_threads(c->nthreads)
  for (int64_t r = 0; r < c->n; ++r) {
    double s = 0.0;
    for (int64_t q = c->rp[r]; q < c->rp[r + 1]; ++q) s += c->v[q] * v[c->ci[q]];
    u[r] = s;
  }
}

/* psi = (A^Pi)^T y = sum_i A_i^T y_i; every column sums its rows in increasing
 * permuted order, i.e. blocks in order and rows in order inside a block. */
static void spmv_t(const orc_ctx *c, const double *y, double *psi) {
#pragma omp parallel for schedule(static) num_threads(c->nthreads)
  for (int64_t k = 0; k < c->n; ++k) {
    double s = 0.0;
    for (int64_t q = c->cp[k]; q < c->cp[k + 1]; ++q) s += c->cv[q] * y[c->ri[q]];
    psi[k] = s;
  }
}

static double dot(int64_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* ===================== exported API ===================== */

void orc_free(orc_ctx *c) {
  if (!c) return;
  free(c->rp0); free(c->ci0); free(c->v0);
  free(c->rp); free(c->ci); free(c->v); free(c->d); free(c->perm); free(c->bp);
  free(c->cp); free(c->ri); free(c->cv);
  free(c->crp); free(c->cci); free(c->ccv);
  free(c->foff); free(c->L);
  free(c->rfoff); free(c->rL);
  free(c->rs); free(c->cs); free(c->ve);
  free(c);
}

/* Build everything the solve needs: copy A, equilibrate rows and columns for
 * ruiz sweeps (0 = off), scale rows to unit 2-norm, permute rows by perm (NULL =
 * identity), column copy, C = A A^T, Gram blocks and their Cholesky factors.
 * factor=0 skips the factorisation (graph-only use).  With equilibration the
 * projections and the CG iterates live in the column-scaled space y = diag(cs) x;
 * orc_solve and orc_cimmino_sweeps return x. */
int orc_setup(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int32_t K,
              const int32_t *perm, const int64_t *bp, int32_t ruiz, int factor, int nthreads,
              orc_ctx **out) {
  *out = NULL;
  if (n <= 0 || K <= 0 || !rp || !ci || !v || !bp || ruiz < 0) return ORC_EINVAL;
  if (bp[0] != 0 || bp[K] != n) return ORC_EINVAL;
  for (int32_t b = 0; b < K; ++b)
    if (bp[b + 1] <= bp[b]) return ORC_EINVAL;
  orc_ctx *c = (orc_ctx *)xcalloc(1, sizeof(orc_ctx));
  if (!c) return ORC_ENOMEM;
  c->n = n;
  c->nnz = rp[n];
  c->K = K;
  c->fail_block = -1;
  c->ruiz = ruiz;
  c->nthreads = nthreads > 0 ? nthreads : 1;
  c->rp0 = (int64_t *)xcalloc(n + 1, sizeof(int64_t));
  c->ci0 = (int32_t *)xcalloc(c->nnz, sizeof(int32_t));
  c->v0 = (double *)xcalloc(c->nnz, sizeof(double));
  c->perm = (int32_t *)xcalloc(n, sizeof(int32_t));
  c->bp = (int64_t *)xcalloc((size_t)K + 1, sizeof(int64_t));
  if (!c->rp0 || !c->ci0 || !c->v0 || !c->perm || !c->bp) { orc_free(c); return ORC_ENOMEM; }
  memcpy(c->rp0, rp, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(c->ci0, ci, sizeof(int32_t) * (size_t)c->nnz);
  memcpy(c->v0, v, sizeof(double) * (size_t)c->nnz);
  memcpy(c->bp, bp, sizeof(int64_t) * (size_t)(K + 1));
  for (int64_t r = 0; r < n; ++r) c->perm[r] = perm ? perm[r] : (int32_t)r;
  int st = equilibrate(c);
  if (st == ORC_OK) st = scale_permute(c);
  if (st == ORC_OK) st = transpose(c);
  if (st == ORC_OK) st = aat(c);
  if (st == ORC_OK && factor) st = factor_all(c);
  *out = c;
  return st;
}

int32_t orc_fail_block(const orc_ctx *c) { return c->fail_block; }

/* The same Gram-block Cholesky as the full setup, for the blocks [b0, b1) only, into
 * storage of their own (replacing an earlier range); OpenMP over the blocks.  With
 * orc_solve_range this times a bounded sample of the setup and of one projection's
 * inner solves on problems whose full oracle run would take too long. */
int orc_factor_range(orc_ctx *c, int32_t b0, int32_t b1) {
  if (!c || b0 < 0 || b1 > c->K || b1 <= b0) return ORC_EINVAL;
  free(c->rfoff); free(c->rL);
  c->rfoff = (int64_t *)xcalloc((size_t)(b1 - b0) + 1, sizeof(int64_t));
  if (!c->rfoff) return ORC_ENOMEM;
  for (int32_t b = b0; b < b1; ++b) {
    int64_t m = c->bp[b + 1] - c->bp[b];
    c->rfoff[b - b0 + 1] = c->rfoff[b - b0] + m * (m + 1) / 2;
  }
  c->rL = (double *)xcalloc((size_t)c->rfoff[b1 - b0], sizeof(double));
  if (!c->rL) return ORC_ENOMEM;
  c->rb0 = b0;
  c->rb1 = b1;
  int fail = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(c->nthreads)
  for (int32_t b = b0; b < b1; ++b) {
    double *L = c->rL + c->rfoff[b - b0];
    gram_block(c, b, L);
    if (cholesky_packed(c->bp[b + 1] - c->bp[b], L) != 0) {
#pragma omp critical
      { fail = 1; }
    }
  }
  return fail ? ORC_ESINGULAR : ORC_OK;
}

/* y_i = G_i^{-1} u_i for the blocks of the last orc_factor_range (u, y: permuted-row
 * n-vectors; rows of other blocks are left untouched). */
int orc_solve_range(const orc_ctx *c, const double *u, double *y) {
  if (!c || !c->rL) return ORC_EINVAL;
#pragma omp parallel for schedule(dynamic, 1) num_threads(c->nthreads)
  for (int32_t b = c->rb0; b < c->rb1; ++b) {
    int64_t r0 = c->bp[b], m = c->bp[b + 1] - r0;
    chol_solve(m, c->rL + c->rfoff[b - c->rb0], u + r0, y + r0);
  }
  return ORC_OK;
}
int64_t orc_aat_nnz(const orc_ctx *c) { return c->nnzc; }

void orc_aat_get(const orc_ctx *c, int64_t *rp, int32_t *ci, double *v) {
  memcpy(rp, c->crp, sizeof(int64_t) * (size_t)(c->n + 1));
  memcpy(ci, c->cci, sizeof(int32_t) * (size_t)c->nnzc);
  memcpy(v, c->ccv, sizeof(double) * (size_t)c->nnzc);
}

void orc_scaled_get(const orc_ctx *c, int64_t *rp, int32_t *ci, double *v, double *d) {
  memcpy(rp, c->rp, sizeof(int64_t) * (size_t)(c->n + 1));
  memcpy(ci, c->ci, sizeof(int32_t) * (size_t)c->nnz);
  memcpy(v, c->v, sizeof(double) * (size_t)c->nnz);
  memcpy(d, c->d, sizeof(double) * (size_t)c->n);
}

/* the equilibration factors: A = diag(rs) Ae diag(cs) (all ones when off) */
void orc_equil_get(const orc_ctx *c, double *rs, double *cs) {
  memcpy(rs, c->rs, sizeof(double) * (size_t)c->n);
  memcpy(cs, c->cs, sizeof(double) * (size_t)c->n);
}

/* dense m x m row-major copy of block b's factor L (upper part zero) */
void orc_factor_get(const orc_ctx *c, int32_t b, double *Ld) {
  int64_t m = c->bp[b + 1] - c->bp[b];
  const double *L = c->L + c->foff[b];
  memset(Ld, 0, sizeof(double) * (size_t)(m * m));
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j <= i; ++j) Ld[i * m + j] = L[pk(i, j)];
}

/* dense m x m row-major copy of block b's Gram matrix G_b (both triangles) */
void orc_gram_get(const orc_ctx *c, int32_t b, double *Gd) {
  int64_t r0 = c->bp[b], r1 = c->bp[b + 1], m = r1 - r0;
  memset(Gd, 0, sizeof(double) * (size_t)(m * m));
  for (int64_t i = r0; i < r1; ++i)
    for (int64_t q = c->crp[i]; q < c->crp[i + 1]; ++q) {
      int64_t j = c->cci[q];
      if (j >= r0 && j < r1) Gd[(i - r0) * m + (j - r0)] = c->ccv[q];
    }
}

/* psi = H v = sum_i A_i^T G_i^{-1} A_i v  (Eq. 1.5); v, psi in column space */
void orc_project(const orc_ctx *c, const double *v, double *psi) {
  double *u = (double *)xcalloc(c->n, sizeof(double));
  double *y = (double *)xcalloc(c->n, sizeof(double));
  spmv(c, v, u);
  block_solves(c, u, y);
  spmv_t(c, y, psi);
  free(u); free(y);
}

/* xi = sum_i A_i^+ f_i with f in the original row order (scaled and permuted here) */
void orc_project_rhs(const orc_ctx *c, const double *f, double *xi) {
  double *fs = (double *)xcalloc(c->n, sizeof(double));
  double *y = (double *)xcalloc(c->n, sizeof(double));
  for (int64_t r = 0; r < c->n; ++r) fs[r] = f[c->perm[r]] / c->d[r];
  block_solves(c, fs, y);
  spmv_t(c, y, xi);
  free(fs); free(y);
}

/* true residual of the original system: ||f - A x||_2, ||.||_inf and gamma (Eq. 3.1) */
static void true_residual(const orc_ctx *c, const double *f, const double *x, double *nrm2,
                          double *gamma) {
  double s2 = 0.0, rinf = 0.0, ainf = 0.0, x1 = 0.0, finf = 0.0;
  for (int64_t i = 0; i < c->n; ++i) {
    double ax = 0.0, arow = 0.0;
    for (int64_t q = c->rp0[i]; q < c->rp0[i + 1]; ++q) {
      ax += c->v0[q] * x[c->ci0[q]];
      arow += fabs(c->v0[q]);
    }
    double r = f[i] - ax;
    s2 += r * r;
    if (fabs(r) > rinf) rinf = fabs(r);
    if (arow > ainf) ainf = arow;
    if (fabs(f[i]) > finf) finf = fabs(f[i]);
    x1 += fabs(x[i]);
  }
  *nrm2 = sqrt(s2);
  double den = ainf * x1 + finf;
  *gamma = den > 0.0 ? rinf / den : 0.0;
}

/* Algorithm 2: CG on H x = xi from x^(0) = 0.  The iteration count is the
 * number of projection sums H p evaluated (xi excluded).  Stops as soon as the
 * true relative residual ||f - A x||_2/||f||_2 <= tol after the x update.
 * hist (optional, maxit entries) receives the relative residual per iteration. */
int orc_solve(const orc_ctx *c, const double *f, double tol, int32_t maxit, double *x,
              int32_t *iters, double *relres, double *gamma, double *hist) {
  int64_t n = c->n;
  double nf = sqrt(dot(n, f, f));
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  *iters = 0;
  *relres = 0.0;
  *gamma = 0.0;
  if (!(nf > 0.0)) return ORC_OK; /* f = 0: x = 0 is exact */
  double *r = (double *)xcalloc(n, sizeof(double));
  double *p = (double *)xcalloc(n, sizeof(double));
  double *psi = (double *)xcalloc(n, sizeof(double));
  double *y = (double *)xcalloc(n, sizeof(double)); /* iterate of A diag(1/cs) y = f */
  orc_project_rhs(c, f, r); /* r^(0) = xi - H y^(0) = xi */
  memcpy(p, r, sizeof(double) * (size_t)n);
  double rho = dot(n, r, r);
  int st = ORC_ENOCONV;
  for (int32_t t = 0; t < maxit; ++t) {
    orc_project(c, p, psi);
    double pq = dot(n, p, psi);
    if (!(pq > 0.0) || !isfinite(pq)) { st = ORC_EBREAKDOWN; *iters = t + 1; break; }
    double alpha = rho / pq;
    for (int64_t i = 0; i < n; ++i) y[i] += alpha * p[i];
    for (int64_t i = 0; i < n; ++i) r[i] -= alpha * psi[i];
    double rho1 = dot(n, r, r);
    double beta = rho1 / rho;
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    rho = rho1;
    for (int64_t i = 0; i < n; ++i) x[i] = c->ruiz > 0 ? y[i] / c->cs[i] : y[i];
    double nr;
    true_residual(c, f, x, &nr, gamma);
    *relres = nr / nf;
    *iters = t + 1;
    if (hist) hist[t] = *relres;
    if (*relres <= tol) { st = ORC_OK; break; }
  }
  if (st == ORC_EBREAKDOWN)
    for (int64_t i = 0; i < n; ++i) x[i] = c->ruiz > 0 ? y[i] / c->cs[i] : y[i];
  free(r); free(p); free(psi); free(y);
  return st;
}

/* Algorithm 1: block Cimmino, x^(t+1) = x^(t) + omega * sum_i A_i^+ (f_i - A_i x^(t)),
 * from x^(0) = 0 for a fixed number of sweeps. */
void orc_cimmino_sweeps(const orc_ctx *c, const double *f, double omega, int32_t sweeps, double *x) {
  int64_t n = c->n;
  double *res = (double *)xcalloc(n, sizeof(double));
  double *y = (double *)xcalloc(n, sizeof(double));
  double *delta = (double *)xcalloc(n, sizeof(double));
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  for (int32_t t = 0; t < sweeps; ++t) {
    /* r_i = f_i - A_i x in the scaled permuted rows */
    for (int64_t r = 0; r < n; ++r) {
      double s = 0.0;
      for (int64_t q = c->rp[r]; q < c->rp[r + 1]; ++q) s += c->v[q] * x[c->ci[q]];
      res[r] = f[c->perm[r]] / c->d[r] - s;
    }
    block_solves(c, res, y);
    spmv_t(c, y, delta);
    for (int64_t i = 0; i < n; ++i) x[i] += omega * delta[i];
  }
  /* the sweeps ran on the column-scaled system; return x = y / cs */
  if (c->ruiz > 0)
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] / c->cs[i];
  free(res); free(y); free(delta);
}

/* Eqs. 2.6-2.7: cutsize(Pi) = sum over cut edges of |c_ij| = interIP(Pi); each
 * undirected edge (i<j) counted once; the diagonal is not an edge.  part[i] is the
 * part of row i of the matrix whose C (CSR, both triangles) is given. */
double orc_cutsize(int64_t n, const int64_t *crp, const int32_t *cci, const double *ccv,
                   const int32_t *part) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t q = crp[i]; q < crp[i + 1]; ++q) {
      int64_t j = cci[q];
      if (j > i && part[i] != part[j]) s += fabs(ccv[q]);
    }
  return s;
}

/* Eqs. 2.8-2.9: ip_km = sum of |c_ij| over rows i in part k and j in part m (K x K,
 * row-major, both orders filled, diagonal = in-block sums over i != j). */
void orc_ip_matrix(int64_t n, const int64_t *crp, const int32_t *cci, const double *ccv,
                   const int32_t *part, int32_t K, double *ip) {
  memset(ip, 0, sizeof(double) * (size_t)K * (size_t)K);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t q = crp[i]; q < crp[i + 1]; ++q) {
      int64_t j = cci[q];
      if (j != i) ip[(int64_t)part[i] * K + part[j]] += fabs(ccv[q]);
    }
}

/* Standalone Gustavson C = A A^T on a caller matrix (no scaling, no permutation).
 * Two calls: with ci_out == NULL it returns nnz(C) in *nnzc and fills rp_out. */
int orc_aat_plain(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                  int64_t *rp_out, int32_t *ci_out, double *v_out, int64_t *nnzc) {
  int64_t bp[2] = {0, n};
  orc_ctx *c = NULL;
  int32_t *perm = (int32_t *)xcalloc(n, sizeof(int32_t));
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  /* run the same Gustavson code on the unscaled matrix */
  c = (orc_ctx *)xcalloc(1, sizeof(orc_ctx));
  c->n = n;
  c->nnz = rp[n];
  c->K = 1;
  c->nthreads = 1;
  c->rp = (int64_t *)xcalloc(n + 1, sizeof(int64_t));
  c->ci = (int32_t *)xcalloc(c->nnz, sizeof(int32_t));
  c->v = (double *)xcalloc(c->nnz, sizeof(double));
  c->bp = (int64_t *)xcalloc(2, sizeof(int64_t));
  c->perm = perm;
  memcpy(c->rp, rp, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(c->ci, ci, sizeof(int32_t) * (size_t)c->nnz);
  memcpy(c->v, v, sizeof(double) * (size_t)c->nnz);
  memcpy(c->bp, bp, sizeof(bp));
  int st = transpose(c);
  if (st == ORC_OK) st = aat(c);
  if (st == ORC_OK) {
    *nnzc = c->nnzc;
    if (rp_out) memcpy(rp_out, c->crp, sizeof(int64_t) * (size_t)(n + 1));
    if (ci_out) memcpy(ci_out, c->cci, sizeof(int32_t) * (size_t)c->nnzc);
    if (v_out) memcpy(v_out, c->ccv, sizeof(double) * (size_t)c->nnzc);
  }
  orc_free(c);
  return st;
}

/* Dense Cholesky of a caller matrix (m x m row-major, lower part read); writes the
 * dense lower factor in place (upper part zeroed).  Returns 0 or -(j+1). */
int orc_cholesky_dense(int64_t m, double *A) {
  double *L = (double *)xcalloc((size_t)(m * (m + 1) / 2), sizeof(double));
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j <= i; ++j) L[pk(i, j)] = A[i * m + j];
  int st = cholesky_packed(m, L);
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < m; ++j) A[i * m + j] = j <= i ? L[pk(i, j)] : 0.0;
  free(L);
  return st;
}

/* ---- Section 2.3, dense columns: the graph is built from a sparser copy of A ----
 * t = floor(sqrt(n)) (integer square root).  A column with more than t nonzeros is
 * dense; it keeps its t entries of largest magnitude (equal magnitudes: the lower
 * row index first) and drops the rest.  Other columns are copied.  The output is a
 * CSR of the same shape whose rows keep their column order; it has at most nnz(A)
 * entries, so out_ci / out_v must hold rp[n] entries.  Returns nnz of the output. */
typedef struct { double a; int64_t row; } orc_mag_row;

static int cmp_mag_row(const void *x, const void *y) {
  const orc_mag_row *p = (const orc_mag_row *)x, *q = (const orc_mag_row *)y;
  if (p->a > q->a) return -1;
  if (p->a < q->a) return 1;
  return p->row < q->row ? -1 : (p->row > q->row ? 1 : 0);
}

int64_t orc_sparsify_dense_columns(int64_t n, const int64_t *rp, const int32_t *ci,
                                   const double *v, int64_t *out_rp, int32_t *out_ci,
                                   double *out_v) {
  int64_t t = 0;
  while ((t + 1) * (t + 1) <= n) ++t;
  int64_t nnz = rp[n];
  int64_t *count = (int64_t *)xcalloc(n, sizeof(int64_t));
  char *keep = (char *)xcalloc(nnz, 1);
  for (int64_t q = 0; q < nnz; ++q) count[ci[q]]++;
  for (int64_t q = 0; q < nnz; ++q) keep[q] = 1;
  orc_mag_row *buf = (orc_mag_row *)xcalloc(n, sizeof(orc_mag_row));
  int64_t *where = (int64_t *)xcalloc(n, sizeof(int64_t));
  for (int64_t j = 0; j < n; ++j) {
    if (count[j] <= t) continue;
    /* gather column j: (|a_ij|, i), rows in increasing order */
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
        if (ci[q] == j) { buf[m].a = fabs(v[q]); buf[m].row = i; where[i] = q; ++m; }
    qsort(buf, (size_t)m, sizeof(orc_mag_row), cmp_mag_row);
    for (int64_t k = t; k < m; ++k) keep[where[buf[k].row]] = 0;
  }
  int64_t w = 0;
  out_rp[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
      if (keep[q]) { out_ci[w] = ci[q]; out_v[w] = v[q]; ++w; }
    out_rp[i + 1] = w;
  }
  free(count); free(keep); free(buf); free(where);
  return w;
}
