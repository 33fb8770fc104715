/*
 * cimmino.h -- C ABI of the GB300 (sm_103a) CG-accelerated block Cimmino solver.
 *
 * The library solves a sparse nonsymmetric, nonsingular system A x = f that is
 * split into K block rows A_i (m_i x n, sum m_i = n; the block-row partition of
 * Eq. 1.2).  It runs Algorithm 2 of Torun, Manguoglu and Aykanat, "A Novel
 * Partitioning Method for Accelerating the Block Cimmino Algorithm" (arXiv
 * 1710.07769): classical CG on H x = xi with H = sum_i A_i^+ A_i (Eq. 1.5),
 * A_i^+ = A_i^T (A_i A_i^T)^{-1} (Section 1) and xi = sum_i A_i^+ f_i
 * (Section 1.1), from x^(0) = 0 (Section 3.1).
 *
 * The projections are applied through the Gram blocks G_i = A_i A_i^T, the
 * diagonal blocks of C = A A^T (Section 2.3, whose pattern and |values| are the
 * row inner-product graph of Section 2.1), factorised once as G_i = L_i L_i^T.
 * Rows are first scaled to unit 2-norm (Section 2.1; H does not depend on row
 * scaling) and permuted into block order (A^Pi = P A, Section 2.2; columns keep
 * their order).
 *
 * Conventions for every entry point:
 *  - Return value: CIMMINO_OK (0) or a negative CIMMINO_E* code; the message of
 *    the last failure of a context is available from cimmino_last_error().
 *  - Device pointers refer to the CUDA device that is current when
 *    cimmino_setup() is called; the context stays bound to that device.
 *  - All device work of a context is ordered on opts.stream (a cudaStream_t).
 *    With opts.stream == NULL the context creates, and later destroys, a
 *    non-blocking stream of its own.  Every call returns after its results are
 *    complete, i.e. calls synchronise that stream before returning.
 *  - A context may be used by one host thread at a time.  Independent contexts
 *    may be used concurrently; the only state they share is the library's
 *    per-device memory pool (see cimmino_opts.alloc), which is thread-safe.
 */
#ifndef CIMMINO_H
#define CIMMINO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define CIMMINO_OK 0
#define CIMMINO_EINVAL (-1)       /* invalid argument or malformed CSR / partition   */
#define CIMMINO_ENOMEM (-2)       /* device or host allocation failed                */
#define CIMMINO_ESINGULAR (-3)    /* a Gram block is not positive definite in FP64:  */
                                  /* A_i is rank deficient (or a row is zero)        */
#define CIMMINO_ENOCONV (-4)      /* max_iter reached; X holds the last iterate      */
#define CIMMINO_EBREAKDOWN (-5)   /* CG breakdown: p^T H p <= 0 or not finite        */
#define CIMMINO_ETIMEOUT (-6)     /* a device-side wait ran out of its budget        */
#define CIMMINO_ECUDA (-7)        /* a CUDA runtime call failed                      */
#define CIMMINO_EUNSUPPORTED (-8) /* input beyond a documented size limit           */

/* ---- precision of the Gram factors and triangular solves ---- */
#define CIMMINO_FP64 0        /* FP64 factors, FP64 solves, no refinement             */
#define CIMMINO_FP32_REFINE 1 /* FP32 factors and solves with FP32 accumulation, FP64 */
                              /* iterative refinement of every inner solve, FP64       */
                              /* refactorisation of blocks with a poor pivot ratio     */

/* ---- storage of the factors ---- */
#define CIMMINO_LAYOUT_DENSE 0   /* every T x T tile of the lower triangle is stored    */
#define CIMMINO_LAYOUT_SKYLINE 1 /* tile row I stores tiles J0(I)..I, where J0(I) is   */
                                 /* the first tile column holding a nonzero of G_i in  */
                                 /* that tile row; Cholesky fill stays inside this     */
                                 /* envelope, so the factor is exact, not approximate  */

/* A square sparse matrix in CSR form.  Column indices must be sorted strictly
 * increasing inside each row and lie in [0, n).  The arrays are read only and
 * stay owned by the caller; they are copied during cimmino_setup(). */
typedef struct cimmino_csr {
  int64_t n;              /* rows = columns                                         */
  int64_t nnz;            /* = row_ptr[n]                                           */
  const int64_t *row_ptr; /* n + 1 offsets, row_ptr[0] = 0                          */
  const int32_t *col_idx; /* nnz column indices                                     */
  const double *val;      /* nnz values                                             */
  int32_t on_device;      /* 1: the three arrays are device pointers, 0: host       */
} cimmino_csr;

/* Caller-supplied device allocator (opts.alloc / opts.free): alloc returns `bytes` of
 * device memory of the context's device usable in stream order on `stream` (a
 * cudaStream_t), or NULL when it cannot (the call then fails with CIMMINO_ENOMEM); free
 * takes back a pointer alloc returned, with the same size and stream.  `user` is
 * opts.alloc_user.  The library calls them from the thread of the API call. */
typedef void *(*cimmino_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*cimmino_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

typedef struct cimmino_opts {
  int32_t precision;      /* CIMMINO_FP64 (default) or CIMMINO_FP32_REFINE           */
  int32_t layout;         /* CIMMINO_LAYOUT_SKYLINE (default) or _DENSE              */
  int32_t tile;           /* tile edge T of the factor layout: 0 = default (64)      */
  int32_t refine_max;     /* refinement steps per inner solve (default 6)           */
  double refine_tol;      /* stop refining when ||G_i y - u_i||_2 <= refine_tol *   */
                          /* ||u_i||_2 (default 1e-12)                               */
  double pivot_ratio_min; /* FP32 block refactored in FP64 when min_j L_jj^2 /      */
                          /* max_j G_jj < pivot_ratio_min (default 1e-4)            */
  int32_t max_iter;       /* CG iteration limit (default 10000, Section 3.1)        */
  int32_t use_graph;      /* 1 (default): capture CG iterations as a CUDA graph     */
  int32_t check_every;    /* CG iterations between convergence read-backs (def. 8)  */
  int32_t keep_aat;       /* 1: keep C = A A^T for cimmino_get_aat() (default 0)    */
  int32_t refine_relax;   /* 1: relaxed inner tolerance in CG iteration t:          */
                          /* min(1e-6, refine_tol / relres_t), relres_t the true    */
                          /* relative residual of the current x (inexact Krylov    */
                          /* subspace methods); 0 (default): refine_tol throughout  */
  int32_t multi_rhs;      /* 1 (default): with several right-hand sides, groups of  */
                          /* 8 or 16 share every factor tile read (CUDA cores);     */
                          /* 2: the same, with the FP32 blocks of up to 32 tile     */
                          /* rows solved on the tensor cores (groups of 16, 3xTF32 */
                          /* products accumulated in tensor memory, about 3x less   */
                          /* accurate than FP32 FMAs: FP64 refinement may take one */
                          /* more step); 0: one factor pass per right-hand side    */
  int32_t ruiz_sweeps;    /* sweeps of row and column infinity-norm equilibration  */
                          /* before the row 2-norm step (Section 3.1), 0..100;     */
                          /* 0 (default): off.  Column scaling changes H (it acts  */
                          /* as a preconditioner); CG then runs on y = diag(cs) x, */
                          /* and solutions are returned as x                       */
  int32_t time_proj;      /* 1: record CUDA events around every projection launch of */
                          /* the CG iterations for cimmino_proj_timing(); the       */
                          /* iterations are then launched eagerly, not as a graph   */
                          /* (events inside a graph cannot be timed); 0 (default)   */
  void *stream;           /* cudaStream_t for all device work (NULL: own stream);  */
                          /* a caller stream must stay valid until cimmino_free()   */
  cimmino_alloc_fn alloc; /* device memory of the context: NULL (default) takes it   */
  cimmino_free_fn free;   /* from a per-device pool of the library, allocated and    */
  void *alloc_user;       /* freed in stream order on opts.stream (cudaMallocAsync-  */
                          /* style; freed blocks stay in the pool for the next      */
                          /* context, so a new context allocates without cudaMalloc */
                          /* once the pool is warm); set both alloc and free to use */
                          /* the caller's allocator (e.g. a framework's caching     */
                          /* allocator), else EINVAL                                 */
  int32_t tune;           /* 1: time the projection kernel's candidate configurations */
                          /* (factor-tile ring depth; registers for one or two CTAs */
                          /* per SM) on this context's blocks at setup and keep the */
                          /* fastest; 0 (default): deepest ring, one CTA per SM.     */
                          /* Results do not depend on the choice (same arithmetic).  */
  const char *tune_cache; /* NULL, or a text file of tuned configurations keyed by   */
                          /* GPU name, precision and block shape: read before tuning */
                          /* (a hit skips the timing), appended after it             */
} cimmino_opts;

/* Statistics of one right-hand side of one system. */
typedef struct cimmino_stats {
  int32_t status;             /* CIMMINO_OK, _ENOCONV, _EBREAKDOWN, _EINVAL (NaN or */
                              /* Inf in this right-hand side) or _EUNSUPPORTED (its */
                              /* squared 2-norm overflows FP64: entries > ~1e154)   */
  int32_t iters;              /* projection sums H p evaluated (xi excluded)       */
  double rel_res;             /* ||f - A x||_2 / ||f||_2 of the returned x          */
  double backward_err;        /* gamma of Eq. 3.1 for the returned x                */
  int64_t refine_steps_total; /* refinement steps summed over blocks and solves     */
  int32_t refine_steps_max;   /* largest number of steps of one inner solve         */
  int32_t fallbacks;          /* blocks refactored in FP64 (whole context)          */
  double t_setup_ms;          /* scaling, permutation, A^T, C = A A^T, G_i extraction */
  double t_factor_ms;         /* Cholesky of all G_i (including FP64 fallbacks)     */
  double t_solve_ms;          /* this solve: xi plus all CG iterations              */
  int64_t nnz_aat;            /* nnz(C) with opts.keep_aat; 0 otherwise (the setup   */
                              /* then forms only the Gram blocks, nnz_gram entries)  */
  int64_t factor_bytes;       /* bytes of the stored factor tiles (L_II and N_IJ)    */
  int64_t pass_bytes;         /* factor bytes one forward + backward solve streams    */
  int64_t kernel_launches;    /* kernels launched by the setup plus by this solve     */
  double factor_flops;        /* algorithmic flops of the Cholesky of all G_i inside */
                              /* the tile envelope (r^3/3 per diagonal tile, r_I r_K^2 */
                              /* per solved tile, 2 r_I r_J r_K per trailing product) */
  double t_chol_ms;           /* device time of the batched Cholesky launch alone    */
  int64_t nnz_gram;           /* entries of the exact Gram blocks G_i (sum over i)    */
  int32_t proj_slots;         /* factor-tile ring depth of the projection kernel      */
  int32_t proj_ctas_per_sm;   /* CTAs per SM its registers are budgeted for (1 or 2)  */
  int32_t proj_tuned;         /* 0 default, 1 measured at setup, 2 from the cache     */
  int32_t mr_tc_blocks;       /* blocks whose multi-RHS projection (nrhs > 1) runs on  */
                              /* the tensor cores; the others run on CUDA cores      */
  int32_t chol_split_blocks;  /* FP64 Cholesky: blocks shared by two CTAs (the largest */
                              /* ones, when they would set the factorisation time)   */
} cimmino_stats;

typedef struct cimmino_ctx cimmino_ctx;

/* Fill *opts with the defaults listed in cimmino_opts. */
void cimmino_opts_default(cimmino_opts *opts);

/* Set up one system: copy A, scale rows to unit 2-norm (Section 2.1), permute rows
 * by perm (Section 2.2), build A^T, C = A A^T (Section 2.3), the Gram blocks G_i
 * and their Cholesky factors.
 *   A          the matrix (host or device arrays, see cimmino_csr).
 *   K          number of blocks, 1 <= K <= n.
 *   perm       host array of n int32: permuted row r is original row perm[r]
 *              (a permutation of 0..n-1), or NULL for the identity.
 *   block_ptr  host array of K+1 int64 offsets over the permuted rows:
 *              0 = block_ptr[0] < block_ptr[1] < ... < block_ptr[K] = n.
 *   opts       NULL for the defaults.
 *   out        receives the new context (NULL on failure).
 * Errors: EINVAL (malformed input), ESINGULAR (a zero row, or a Gram block that is
 * not positive definite in FP64), EUNSUPPORTED (a block with more than 4096 rows, or
 * a row of C with more than 8192 structural candidates), ENOMEM, ECUDA. */
int cimmino_setup(const cimmino_csr *A, int32_t K, const int32_t *perm, const int64_t *block_ptr,
                  const cimmino_opts *opts, cimmino_ctx **out);

/* Set up a batch of nsys independent systems that are solved together: system s
 * has matrix A[s], K[s] blocks, perm[s] (NULL entry or NULL array = identity) and
 * block_ptr[s].  Every stage runs as one launch over all blocks of all systems. */
int cimmino_setup_batch(int32_t nsys, const cimmino_csr *A, const int32_t *K,
                        const int32_t *const *perm, const int64_t *const *block_ptr,
                        const cimmino_opts *opts, cimmino_ctx **out);

/* Solve A X = F for nrhs right-hand sides of a single-system context
 * (Algorithm 2 per right-hand side, all right-hand sides sharing every pass over
 * A and the factors).
 *   F, X       n x nrhs, column k at F + k*ld (column-major), original row order
 *              for F and original column order for X; X is caller-allocated and
 *              receives the solutions.
 *   on_device  1: F and X are device pointers, 0: host pointers.
 *   tol        stop right-hand side k once ||f_k - A x_k||_2 <= tol * ||f_k||_2.
 *   stats      NULL or an array of nrhs entries.
 * Returns CIMMINO_OK when every right-hand side converged, else the first
 * failure (ENOCONV / EBREAKDOWN; X still holds the last iterates; EINVAL for a
 * right-hand side holding NaN or Inf and EUNSUPPORTED for one whose squared 2-norm
 * overflows FP64, whose x stays 0; the other right-hand sides are still solved). */
int cimmino_solve(cimmino_ctx *ctx, const double *F, int32_t nrhs, int64_t ld, double tol,
                  double *X, int32_t on_device, cimmino_stats *stats);

/* Solve every system of a batch context once: F[s] and X[s] are n_s-vectors
 * (host or device as on_device says); stats NULL or nsys entries. */
int cimmino_solve_batch(cimmino_ctx *ctx, const double *const *F, double tol, double *const *X,
                        int32_t on_device, cimmino_stats *stats);

/* Release a context and all of its device memory.  NULL is allowed. */
void cimmino_free(cimmino_ctx *ctx);

/* Message of the last failure of ctx (or of the last failed setup when ctx is NULL,
 * per host thread).  The string stays valid until the next call on ctx. */
const char *cimmino_last_error(const cimmino_ctx *ctx);

/* ---- inspection hooks (tests, partitioners) ----
 * All copy into caller-allocated HOST buffers. */

/* nnz of C = A A^T of the scaled permuted matrix; then its CSR (columns sorted,
 * structural pattern: entries whose value cancels to 0.0 are kept).  Needs
 * opts.keep_aat = 1 at setup, else EINVAL.  Single-system contexts only. */
int cimmino_get_aat_nnz(cimmino_ctx *ctx, int64_t *nnz);
int cimmino_get_aat(cimmino_ctx *ctx, int64_t *row_ptr, int32_t *col_idx, double *val);

/* Scaled permuted matrix S (CSR, nnz entries) and the row factors d (n), with
 * P A = diag(d) S diag(cs): S has unit 2-norm rows; d is the row 2-norm times the
 * equilibration row divisor, cs the column divisors (cimmino_get_colscale). */
int cimmino_get_scaled(cimmino_ctx *ctx, int64_t *row_ptr, int32_t *col_idx, double *val,
                       double *d);

/* Column equilibration divisors cs (n doubles; all ones with opts.ruiz_sweeps = 0).
 * The projections (cimmino_project, cimmino_project_rhs) act in the column-scaled
 * space y = diag(cs) x.  Errors: EINVAL (NULL pointer), ECUDA. */
int cimmino_get_colscale(cimmino_ctx *ctx, double *cs);

/* Number of rows m of global block b (blocks of all systems in order). */
int cimmino_block_rows(cimmino_ctx *ctx, int32_t b, int32_t *m);

/* Dense m x m row-major copy of the Cholesky factor L_b (upper part zero),
 * converted to double; *is_fp64 tells which precision the block was factored in. */
int cimmino_get_factor(cimmino_ctx *ctx, int32_t b, double *L, int32_t *is_fp64);

/* Projection sums psi_k = H v_k = sum_i A_i^+ A_i v_k (Eq. 1.5), k < nrhs, of a
 * single-system context, with the same kernels (and refinement) as CG iterations
 * with nrhs right-hand sides: for nrhs > 1 and opts.multi_rhs, groups of
 * right-hand sides share every factor tile read.  v and psi are nrhs x n arrays
 * (vector k at offset k * n) in the original column order, host or device memory
 * (copies use unified addressing; on_device is informational).
 * Errors: EINVAL (NULL pointer, nrhs < 1, batch context), ECUDA, ENOMEM. */
int cimmino_project(cimmino_ctx *ctx, const double *v, int32_t nrhs, double *psi,
                    int32_t on_device);

/* xi_k = sum_i A_i^+ f_{k,i} (Section 1.1), k < nrhs, for right-hand sides f in the
 * original row order (nrhs x n, vector k at offset k * n); xi is nrhs x n.
 * Errors as cimmino_project. */
int cimmino_project_rhs(cimmino_ctx *ctx, const double *f, int32_t nrhs, double *xi,
                        int32_t on_device);

/* Standalone C = A A^T of a caller matrix (no scaling, no permutation) on the
 * GPU, e.g. to build the row inner-product graph for a partitioner.  Two calls:
 * first with col_idx = val = NULL to get *nnz and row_ptr (n+1), then with
 * buffers of *nnz entries.  Host buffers.  stream: cudaStream_t or NULL. */
int cimmino_aat(const cimmino_csr *A, void *stream, int64_t *nnz, int64_t *row_ptr,
                int32_t *col_idx, double *val);

/* C = A A^T into caller-owned DEVICE buffers without allocating any device memory.
 * The paper has no counterpart.  Some callers cannot let a library allocate: an
 * embedder whose device memory is all reserved by its own allocator (a framework's
 * caching pool) or capped by a fixed budget would see cudaMalloc fail or exceed that
 * budget, and a latency-bound loop cannot afford cudaMalloc / cudaFree, which may block
 * the host and synchronise the device.  For them this computes the same result as
 * cimmino_aat() (same kernels, bitwise equal) with the working memory taken from a
 * fixed static array instead.
 *   A         device CSR (A->on_device must be 1), n <= 262,144 and nnz <= 2,097,152,
 *             else CIMMINO_EUNSUPPORTED.
 *   stream    cudaStream_t for the work (NULL: legacy default stream).
 *   nnz       host out: nnz(C).
 *   row_ptr   device out, n + 1 entries (always written).
 *   col_idx, val  device out with room for `capacity` entries, or both NULL to only
 *             count (first call of a two-call pattern); EINVAL if capacity < nnz(C).
 * Memory: the working arrays (transpose of A, counts, scan partials) live in one
 * static device array of about 33 MB that every GPU loading this library keeps until
 * the process exits.  No cudaMalloc / cudaFree or allocating library call is made.
 * The first call on each device looks up that array's device address (with the
 * device current) and caches it for the life of the process, so the entry point must
 * not be used on a device after cudaDeviceReset() (or any other re-creation of its
 * primary context) in the same process.  All calls share the array, which keeps the
 * last call's contents: each call clears what must start at zero, and calls whose
 * work overlaps on the GPU (other host threads, other streams) race on the array and
 * must be serialised by the caller.  The call is host-synchronous: it synchronises
 * `stream` between its stages (to read counts back to the host) and before it
 * returns.  The error message is available from cimmino_last_error(NULL). */
int cimmino_aat_noalloc(const cimmino_csr *A, void *stream, int64_t *nnz, int64_t *row_ptr,
                        int32_t *col_idx, double *val, int64_t capacity);

/* Dense columns (Section 2.3): a column with more than sqrt(n) nonzeros would make
 * C = A A^T, and the row inner-product graph, dense.  Writes a copy of A in which every
 * column with more than t = floor(sqrt(n)) nonzeros keeps only its t entries of
 * largest magnitude (equal magnitudes: lower row first); other entries are copied in
 * their row order.  For building the partitioning graph only (cimmino_aat on the copy,
 * then cimmino_partition_rip); the solve uses the full A.  Host-only, no GPU.
 *   n, row_ptr, col_idx, val     host CSR of A (n x n).
 *   out_row_ptr (n + 1), out_col_idx and out_val (row_ptr[n] entries each, the most
 *                                the copy can have): caller-allocated host arrays.
 *   nnz_out                      out: nnz of the copy.
 * Errors: EINVAL (NULL pointer, n < 1, malformed row_ptr, column out of range), ENOMEM. */
int cimmino_sparsify_dense_columns(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                   const double *val, int64_t *out_row_ptr,
                                   int32_t *out_col_idx, double *out_val, int64_t *nnz_out);

/* Block-row partition by the row inner-product graph G_RIP (Sections 2.1-2.3): vertices
 * are rows, edge (i, j) carries cost |c_ij| / sqrt(c_ii c_jj), the cosine of rows i and j
 * after unit 2-norm row scaling, for every nonzero c_ij of C = A A^T.  The K-way
 * partition minimises the cutsize (Eq. 2.6 = sum of inter-block |inner products|) subject
 * to at most `cap` rows per block (Eq. A.1 with unit vertex weights; cap = n / K gives
 * exact balance).  Host-only, no GPU: multilevel heavy-edge coarsening, recursive
 * bisection, balance-constrained k-way refinement; rows inside a block are ordered by
 * reverse Cuthill-McKee (the order inside a block is free, Section 2.2).
 *   C            host CSR of A A^T of the UNSCALED matrix with its diagonal (e.g. from
 *                cimmino_aat); row i needs c_ii > 0.
 *   K, cap       number of blocks (1 <= K <= n) and the row cap (cap * K >= n).
 *   seed         random seed of the matching and bisection orders.
 *   perm         out, n int32: block row order (permuted row r = original row perm[r]).
 *   block_ptr    out, K+1 int64 offsets over the permuted rows.
 *   cutsize      out (may be NULL): cut of the returned partition in cosine units.
 * Errors: EINVAL, ENOMEM. */
int cimmino_partition_rip(int64_t n, const int64_t *crp, const int32_t *cci, const double *ccv,
                          int32_t K, int32_t cap, uint64_t seed, int32_t *perm,
                          int64_t *block_ptr, double *cutsize);

/* The static schedule of the FP64 Cholesky (the batched factorisation of the G_i that the
 * setup runs for FP64 blocks), as a host-only function for inspection and tests; the paper has
 * no counterpart (it factors each block on its own process).  Block b has nt[b] tile rows of
 * 64, ntrsm[b] stored tiles (I, K) below the diagonal (each solved once, with the symmetric
 * update of (I, I)) and nfull[b] full trailing-update tiles (I, J), K < J < I.  Its cost, in
 * units of one full update tile, is 1.41 nt + 0.59 ntrsm + nfull (weights measured on GB300).
 * The blocks are packed onto at most maxcta CTA lists by MULTIFIT (the smallest capacity that
 * first-fit decreasing fills) and a move/swap pass; with allow_split, blocks whose cost
 * reaches 0.9 of the mean load per CTA may be shared by two CTAs (their diagonal tiles on
 * part 0, the rest halved, plus 0.09 per tile row for the pair barriers), the split count
 * chosen from a ladder for the shortest makespan.
 *   ncta        out: lists used (<= maxcta).
 *   cta_ptr     out, ncta + 1 entries (caller array of maxcta + 1): list k is items
 *               cta_ptr[k] .. cta_ptr[k+1] - 1.
 *   items       out, triples (block, part, nparts) (caller array of 3 * (nblk + maxcta / 2));
 *               a split block appears twice (parts 0 and 1, nparts = 2), first in two lists.
 *   nsplit      out: split blocks.  makespan: out, the largest list's cost.
 * Host-only, no GPU.  Errors: EINVAL (nblk < 0, maxcta < 1, NULL pointers, nt < 1 or
 * negative counts), ENOMEM. */
int cimmino_cholesky_schedule(int32_t nblk, const int32_t *nt, const int64_t *ntrsm,
                              const int64_t *nfull, int32_t maxcta, int32_t allow_split,
                              int32_t *ncta, int32_t *cta_ptr, int32_t *items, int32_t *nsplit,
                              double *makespan);

/* Algorithm 1 (Section 1.1): the block Cimmino iteration with relaxation parameter
 * omega, x^(t+1) = x^(t) + omega * sum_i A_i^+ (f_i - A_i x^(t)), from x^(0) = 0, for
 * `sweeps` sweeps, on the same setup (scaling, factors, refinement) as the CG solve.
 * f: nrhs x n right-hand sides in the original row order; x: nrhs x n result in the
 * original column order (vector k at offset k * n); host or device memory.  Block
 * Cimmino converges for 0 < omega < 2 / rho(H) (Section 1.1); no test is applied here.
 * Errors: EINVAL (NULL pointer, nrhs < 1, sweeps < 0, omega not finite, batch
 * context), ECUDA, ENOMEM. */
int cimmino_sweeps(cimmino_ctx *ctx, const double *f, int32_t nrhs, double omega,
                   int32_t sweeps, double *x, int32_t on_device);

/* Benchmark hook: after a cimmino_solve() on a single-system context, launch each
 * per-iteration kernel `reps` times back to back on the context's stream, on the
 * vectors of the last solve, and write the average device time per launch in
 * milliseconds (CUDA events recorded on that stream):
 *   ms[0] projection kernel y_i = G_i^{-1} u_i over all blocks (with refinement in
 *         FP32 mode), ms[1] u = A p, ms[2] psi = A^T y.
 * ms is a caller array of 3 doubles.  Errors: EINVAL (no solve yet, reps < 1). */
int cimmino_time_kernels(cimmino_ctx *ctx, int32_t reps, double *ms);

/* Benchmark hook: device time of the projection launches inside the CG iterations of
 * the last cimmino_solve() / cimmino_solve_batch() on a context set up with
 * opts.time_proj = 1, measured live in the iteration sequence (CUDA events recorded on
 * the context's stream before and after each projection launch).  Only the launches of
 * iterations in which some lane was still running count (the projections that produced
 * the returned x).  *ms_total receives their summed milliseconds, *launches their number.
 * Errors: EINVAL (NULL pointer, time_proj off, no solve yet). */
int cimmino_proj_timing(cimmino_ctx *ctx, double *ms_total, int64_t *launches);

/* Watchdog self-test (failure detection without a GPU fault): one device thread waits,
 * with the same bounded try_wait loop as the projection ring, on an mbarrier that nothing
 * completes.  After limit_us microseconds (or 2^20 polls) it gives up and sets bit 8 of
 * the device error word.  Then a CTA waits, as one half of a block the FP64 Cholesky splits
 * over two CTAs, for a partner that never arrives (a flag nothing sets); it gives up after
 * limit_us and sets bit 16.  The word is copied to *err_word (24 when both gave up).  Needs
 * no context; runs on a stream of its own on the current device.
 * Returns CIMMINO_ETIMEOUT when the wait gave up (the expected outcome), CIMMINO_OK if
 * it did not, EINVAL (limit_us outside [1, 1e6], NULL err_word), ECUDA, ENOMEM. */
int cimmino_selftest_wait(int32_t limit_us, int32_t *err_word);

/* Benchmark hook: the FP64 FMA rate of the current device in TFLOP/s (2 flops per FMA),
 * measured by a kernel of independent FMA chains on every SM (CUDA events, after a warm-up
 * launch).  It is the ALU roofline of the FP64 kernels, which GB300's FP64 pipe bounds.
 * Errors: EINVAL (NULL), ECUDA, ENOMEM. */
int cimmino_fp64_peak(double *tflops);

/* Library build information (compile-time architecture, version). */
const char *cimmino_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CIMMINO_H */
