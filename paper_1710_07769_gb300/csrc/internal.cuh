// Internal declarations of the GB300 block Cimmino library (not part of the C ABI).
//
// Data layout in HBM (all systems of a batch concatenated into one block-diagonal
// matrix, so every stage is a single launch over all rows / blocks):
//   A     : scaled, permuted CSR  (rp int64 [N+1], ci int32 [nnz], va f64 [nnz])
//   At    : its transpose (CSC of A), rows increasing inside a column
//   d     : row 2-norms of the original rows, permuted order
//   C_bd  : block-diagonal part of C = A A^T: CSR over global rows with column
//           indices local to the block (int32) and FP64 values -- the exact G_i,
//           used by the FP64 refinement residual and to rebuild G_i for fallbacks
//   factors: per block, per tile row I, the T x T tiles J0(I)..I of L_i stored
//           contiguously (row-major inside a tile); dinv holds inv(L_II) per tile row.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/cimmino.h"

namespace cimmino {

constexpr int kTile = 64;          // tile edge T of the factor layout
constexpr int kMaxBlockRows = 4096;
constexpr int kSpgemmWarpCap = 1024;   // candidates per row handled by one warp
constexpr int kSpgemmCtaCap = 8192;    // candidates per row handled by one CTA
constexpr int kMaxProjSlots = 16;      // factor-tile slots of the projection kernel's ring
constexpr int kVecRows = 256;          // rows (= threads) per CTA of the CG vector kernels
constexpr int kProjSmemMax = 231424;   // dynamic shared memory budget of one projection CTA
// Packed triangular tiles (rectangular full packed): row pair p = 0..31 holds the entries of
// rows p and 63 - p of a lower (or upper) triangular 64 x 64 tile, 65 values, padded to 68.
constexpr int kPackPair = 68;
constexpr int kPackTile = 32 * kPackPair;  // 2176 entries instead of 4096
// Block-packed triangular tiles (FP32): row pair p holds the 16-wide sub-tile segments of
// rows p and 63 - p inside the triangle, 5 segments = 80 values, padded to 84.
constexpr int kBPackPair = 84;
constexpr int kBPackTile = 32 * kBPackPair;  // 2688 entries instead of 4096

struct BlockDesc {
  int64_t row0;      // first global (permuted, concatenated) row
  int64_t dinv_off;  // element offset of this block's inv(L_II) tiles in its dinv array
  int32_t m;         // rows of the block
  int32_t nt;        // tile rows = ceil(m / T)
  int32_t trow0;     // first entry of this block in the tile-row table
  int32_t sys;       // system index
  int32_t prec64;    // 1: factor stored in FP64 arrays, 0: FP32 arrays
  int32_t slice0;    // first 32-row slice of this block in the sliced-ELL Gram copy
};

struct TileRow {
  int64_t off;  // element offset of tile (I, J0) in the factor array of the block
  int32_t j0;   // first stored tile column J0(I)
  int32_t pad;
};

struct SysDesc {
  int64_t row0;  // first global row (and column) of the system
  int64_t n;     // rows of the system
  int32_t cta0;  // first CTA of the system in the vector-kernel CTA table
  int32_t ncta;  // CTAs of the system
};

// CTA table of the vector kernels: every CTA covers rows of exactly one system,
// so per-CTA partial sums belong to one lane and are reduced in a fixed order.
struct CtaDesc {
  int64_t row0;
  int32_t rows;
  int32_t sys;
  int32_t slice0;  // first 32-row slice of the CTA in the sliced-ELL copies of A and A^T
  int32_t pad;
};

// Per right-hand side of a system ("lane") CG state, written by the kernels.
struct LaneState {
  double fnorm2;   // ||f||_2^2 of the original right-hand side
  double rho[2];   // r^T r, indexed by iteration parity
  double alpha;
  double beta;
  double pq;       // p^T H p of the current iteration
  double relres;   // true relative residual of the current x
  int32_t status;  // 0 running, 1 converged, CIMMINO_ENOCONV, CIMMINO_EBREAKDOWN
  int32_t iters;   // projections used to produce the current x
  int32_t t;       // iteration counter
  int32_t pad;
};

#define CIMMINO_RUNNING 0
#define CIMMINO_CONVERGED 1

// --------------------------------------------------------------------------
// host-side error handling
struct Error {
  int code;
  std::string msg;
};

#define CUDA_TRY(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess)                                                    \
      throw ::cimmino::Error{CIMMINO_ECUDA, std::string(#call) + ": " +      \
                                                cudaGetErrorString(e_)};      \
  } while (0)

inline void fail(int code, const std::string &msg) { throw Error{code, msg}; }

// Sets the per-thread message returned by cimmino_last_error(NULL) (defined in api.cu).
void record_last_error(const std::string &msg);

// --------------------------------------------------------------------------
// device helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic CTA-wide sum (fixed tree); every thread gets the result.
// scratch: >= 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double *scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double t = (threadIdx.x < (unsigned)nw) ? scratch[threadIdx.x] : 0.0;
  if (warp == 0) t = warp_sum(t);
  if (threadIdx.x == 0) scratch[0] = t;
  __syncthreads();
  double r = scratch[0];
  __syncthreads();
  return r;
}

// --------------------------------------------------------------------------
// launchers (defined in the .cu files)

// setup_kernels.cu
void launch_check_perm(const int32_t *perm, int64_t n, int32_t *seen, int32_t *flag,
                       cudaStream_t s);
void launch_validate_csr(const int64_t *rp, const int32_t *ci, int64_t n, int64_t nnz,
                         int32_t *flag, cudaStream_t s);
int64_t scan_tmp_len(int64_t n);
void launch_scan_counts(const int64_t *counts, int64_t *out, int64_t n, int64_t *tmp,
                        int64_t tmp_len, cudaStream_t s);
void launch_permuted_lengths(const int64_t *rp0, const int32_t *perm, int64_t N, int64_t *len,
                             cudaStream_t s);
// Section 3.1 equilibration, in place on v (pattern rp/ci): `sweeps` sweeps of
// row and column infinity-norm scaling; rs / cs receive the accumulated divisors
// (A = diag(rs) Ae diag(cs)).  work: 3 N doubles of scratch.
void launch_equilibrate(const int64_t *rp, const int32_t *ci, double *v, int64_t N,
                        int32_t sweeps, double *rs, double *cs, double *work, cudaStream_t s);
void launch_scale_permute(const int64_t *rp0, const int32_t *ci0, const double *v0,
                          const int32_t *perm, const int64_t *rp, int64_t N, int32_t *ci,
                          double *va, double *d, const double *rs, int32_t *flag, cudaStream_t s);
void launch_transpose(const int64_t *rp, const int32_t *ci, const double *va, int64_t N,
                      int64_t nnz, int64_t *cp, int32_t *ri, double *cv, int64_t *work,
                      int64_t *tmp, int64_t tmp_len, cudaStream_t s);
// C = A A^T by rows.  With blk and rowblk (row -> block), row i keeps only the columns of its
// own block (the Gram block G_i, global column indices); without them, every column.
void spgemm_count(const int64_t *rp, const int32_t *ci, const int64_t *cp, const int32_t *ri,
                  int64_t N, int64_t *cnt, int32_t *ovf, int32_t *ovf_n, cudaStream_t s,
                  const BlockDesc *blk = nullptr, const int32_t *rowblk = nullptr);
void spgemm_overflow(const int64_t *rp, const int32_t *ci, const double *va, const int64_t *cp,
                     const int32_t *ri, const int32_t *ovf, int32_t novf, int64_t *cnt,
                     const int64_t *crp, int32_t *cci, double *ccv, int32_t *flag,
                     cudaStream_t s, const BlockDesc *blk = nullptr,
                     const int32_t *rowblk = nullptr);
// cv: values of the transpose (CSC of A), aligned with ri
void spgemm_fill(const int64_t *rp, const int32_t *ci, const double *va, const int64_t *cp,
                 const int32_t *ri, const double *cv, int64_t N, const int64_t *crp,
                 int32_t *cci, double *ccv, cudaStream_t s, const BlockDesc *blk = nullptr,
                 const int32_t *rowblk = nullptr);
// block-restricted rows of C: global columns -> block-local ones, and each row's first one
void bd_localize(const int64_t *brp, int32_t *bci, const BlockDesc *blk, const int32_t *rowblk,
                 int64_t N, int32_t *rowmin, cudaStream_t s);
void launch_row_block_ids(const BlockDesc *blk, int32_t nblk, int32_t *rowblk, cudaStream_t s);
void bd_count(const int64_t *crp, const int32_t *cci, const BlockDesc *blk, const int32_t *rowblk,
              int64_t N, int64_t *cnt, cudaStream_t s);
void bd_fill(const int64_t *crp, const int32_t *cci, const double *ccv, const BlockDesc *blk,
             const int32_t *rowblk, int64_t N, const int64_t *brp, int32_t *bci, double *bcv,
             int32_t *rowmin, cudaStream_t s);
void launch_tile_j0(const BlockDesc *blk, int32_t nblk, const int32_t *rowmin, int dense,
                    int32_t *j0, cudaStream_t s);
void sell_width(const BlockDesc *blk, int32_t nblk, const int64_t *brp, int64_t *cnt,
                cudaStream_t s);
void sell_fill(const BlockDesc *blk, int32_t nblk, const int64_t *brp, const int32_t *bci,
               const double *bcv, const int64_t *soff, int16_t *scol, double *sval,
               cudaStream_t s);
// rows of every CTA-table chunk by decreasing length (ord[position] = row)
void chunk_order(const int64_t *ptr, const CtaDesc *cta, int32_t ncta, int32_t *ord,
                 cudaStream_t s);
// sliced-ELL copy of a CSR matrix; rmap (optional) gives the row at each position
void sell_rows_width(const int64_t *ptr, const int64_t *srow0, const int32_t *srows,
                     int32_t nslice, const int32_t *rmap, int64_t *cnt, cudaStream_t s);
void sell_rows_fill(const int64_t *ptr, const int32_t *idx, const double *val,
                    const int64_t *srow0, const int32_t *srows, int32_t nslice,
                    const int32_t *rmap, const int64_t *off, int32_t *ocol, double *oval,
                    cudaStream_t s);
void launch_gram_scatter(const BlockDesc *blk, const int32_t *blist, int32_t nlist,
                         const TileRow *trow, const int64_t *brp, const int32_t *bci,
                         const double *bcv, void *fac, int64_t fac_elems, int prec64,
                         cudaStream_t s);

// factor arrays of both precisions (a context may hold FP64 fallback blocks beside
// FP32 blocks): forward tiles (L_II, N_IJ), inv(L_II), and their transposed copies
struct FactorPtrs {
  const float *fac32;
  const float *dinv32;
  float *facT32;
  float *dinvT32;
  const double *fac64;
  const double *dinv64;
  double *facT64;
  double *dinvT64;
  double *dinvP64;   // packed inv(L_II) (lower) and inv(L_II)^T (upper) of FP64 blocks,
  double *dinvTP64;  // kPackTile entries per tile
  float *dinvP32;    // block-packed ones of FP32 blocks, kBPackTile entries per tile
  float *dinvTP32;
};

// chol_tc.cu: FP32 blocks, left-looking on the tensor cores (tcgen05, 3xTF32), then the N
// transform of every off-diagonal tile.  scratch: cholesky_tc_scratch_floats(factor elements)
// floats (the split operand copy of L and a zero image); rowblk_t: one int per tile row.
int64_t cholesky_tc_scratch_floats(int64_t factor_elems);
void launch_cholesky_tc(const BlockDesc *blk, const int32_t *blist, int32_t nlist, int32_t nblk,
                        int32_t ntrow, const TileRow *trow, float *fac, float *dinv,
                        float *scratch, int64_t factor_elems, int32_t *rowblk_t, double *pivmin,
                        int32_t *pivfail, int32_t *err, cudaStream_t s);
// the same for the FP32 blocks (all tile rows of the context; rowblk_t: ntrow scratch)
void launch_ntransform_tc(const BlockDesc *blk, int32_t nblk, int32_t ntrow, const TileRow *trow,
                          float *fac, const float *dinv, int32_t *rowblk_t, cudaStream_t s);

// chol_kernels.cu
void launch_transpose_factor(const BlockDesc *blk, int32_t nblk, const TileRow *trow,
                             const TileRow *trowT, const FactorPtrs &f, cudaStream_t s);
// FP64 blocks (FP64 precision and the FP64 refactorisation of FP32 blocks) on a static
// schedule: CTA c factors items[cta_ptr[c] .. cta_ptr[c + 1]).  An item with nparts = 2 is half
// of a block shared by two CTAs, which meet through pair_flags[2 slot], [2 slot + 1] (zeroed
// before the launch); such a schedule needs all its CTAs resident at once and is launched
// cooperatively (ncta <= cholesky_resident_ctas()).  A pair wait that runs out after ~2 s sets
// *err.
struct CholItem {
  int32_t b;       // block
  int32_t part;    // 0 or 1 of a split block
  int32_t nparts;  // 1, or 2 for a split block
  int32_t slot;    // pair-flag slot of a split block
};
int32_t cholesky_resident_ctas();
// watchdog self-test of the pair wait (flag: two zeroed ints; sets bit 16 of *err)
void launch_pair_selftest(uint64_t limit_ns, int32_t *flag, int32_t *err, cudaStream_t s);
cudaError_t launch_cholesky(const BlockDesc *blk, const CholItem *items, const int32_t *cta_ptr,
                            int32_t ncta, bool cooperative, const TileRow *trow, double *fac,
                            double *dinv, double *pivmin, int32_t *pivfail, int32_t *pair_flags,
                            int32_t *err, cudaStream_t s);
// N_KJ = inv(L_KK) L_KJ for the off-diagonal tiles of the listed FP64 blocks (after the Cholesky)
void launch_ntransform64(const BlockDesc *blk, const int32_t *blist, int32_t nlist,
                         const TileRow *trow, double *fac, const double *dinv, cudaStream_t s);

// solve_kernels.cu
struct IterArgs {
  const int64_t *rp;
  const int32_t *ci;
  const double *va;
  const int64_t *cp;
  const int32_t *ri;
  const double *cv;
  const double *d;
  const double *cs;  // column equilibration divisors (x = y / cs), nullptr when off
  const int64_t *brp;
  const int32_t *bci;
  const double *bcv;
  const int64_t *aoff;   // sliced-ELL copy of A (32-row slices, [k][lane]): offsets
  const int32_t *acol;   //   columns
  const double *aval;    //   values
  const int64_t *toff;   // sliced-ELL copy of A^T (32-column slices)
  const int32_t *tord;   //   the column of A^T at each position (sorted inside CTA chunks)
  const int32_t *tcol;   //   rows
  const double *tval;    //   values
  const int64_t *soff;   // sliced-ELL Gram blocks: slice offsets (entries)
  const int16_t *scol;   //   block-local columns
  const double *sval;    //   values
  const BlockDesc *blk;
  const int32_t *border;  // launch order of the blocks in the projection kernels: most
                          // streamed tiles first, so that the long ones start in wave one
  const TileRow *trow;
  const TileRow *trowT;  // upper (transposed) tile rows: off, j0 field = J1(I)
  const float *fac32;
  const float *dinv32;
  const float *facT32;
  const float *dinvT32;
  const double *fac64;
  const double *dinv64;
  const double *facT64;
  const double *dinvT64;
  const double *dinvP64;  // packed triangular inv(L_II), inv(L_II)^T of FP64 blocks
  const double *dinvTP64;
  const float *dinvP32;   // block-packed ones of FP32 blocks
  const float *dinvTP32;
  const SysDesc *sys;
  const CtaDesc *cta;
  LaneState *lane;
  double *fs;     // scaled permuted right-hand sides, [N][nrhs] (row space)
  double *x;      // [N][nrhs] (column space)
  double *p;
  double *r;
  double *psi;
  double *u;      // [N][nrhs] (row space)
  double *y;
  double *part;   // partial sums: 4 kinds x [ncta][nrhs]
  int32_t *cnt;   // last-CTA arrival counters: 4 kinds x nsys
  int64_t *refine_total;
  int32_t *refine_max;
  int64_t N;
  int32_t nsys;
  int32_t ncta;
  int32_t nblk;
  int32_t nrhs;
  int32_t refine_steps;  // refinement steps allowed per inner solve of FP32 blocks
  int32_t max_mp;        // largest padded block (rows), sizes the projection smem
  int32_t proj_smem;     // dynamic shared memory bytes of the projection kernel
  int32_t proj_slots;    // factor-tile slots in the projection kernel's ring
  int32_t proj_minb;     // CTAs per SM the projection kernel is compiled for (1 or 2)
  int32_t proj_slot_bytes;
  int32_t proj_wbytes;   // bytes per entry of the projection's working vectors (4 or 8)
  int32_t proj_rg;       // right-hand sides per group of the multi-RHS projection (0: off)
  int32_t proj_mr_slots; // factor-tile slots of the multi-RHS projection's ring
  int32_t proj_mr_smem;  // dynamic shared memory bytes of the multi-RHS projection
  const int32_t *mr_list;  // multi-RHS launch order: tensor-core blocks first, then the rest
  int32_t mr_ntc;          // blocks at the front of mr_list taken by the tensor-core kernel
  const void *mr_tmaps;    // host array of 4 tensor maps (fac32, facT32, dinv32, dinvT32)
  int32_t *err;          // device error word: bounded waits that ran out
  int32_t max_iter;
  int32_t refine_relax;  // 1: inner tolerance min(1e-6, refine_tol / relres_t) in iterations
  double refine_tol;
  double tol;
};

// Inner-solve tolerance of lane `l` (relative ||G y - u|| / ||u||).  With refine_relax, a
// projection inside CG iteration t may be as inexact as refine_tol / relres_t, where
// relres_t is the true relative residual of the current iterate: the inexact-Krylov
// bound lets the error of the operator application grow as the residual shrinks.  The
// 1e-6 cap keeps it at the FP32 solve's own accuracy.  Outside iterations (check_lane 0:
// the right-hand side projection and the inspection hooks) refine_tol applies.
__device__ __forceinline__ double inner_tol(const IterArgs &a, int check_lane, int64_t l) {
  if (!a.refine_relax || !check_lane) return a.refine_tol;
  const double rr = a.lane[l].relres;
  return fmin(1e-6, a.refine_tol / fmax(rr, 1e-300));
}

// FP64 refinement residual of row r (block-local) for a group of RG right-hand sides:
// acc[g] -= sum_c G_rc y[c][g] over the row's entries in the sliced-ELL Gram copy (in entry
// order), for the active g (bit g of mask).  y rows are [ld] doubles, the group at column k0.
// A full group with an even row length reads each y row as 16-byte pairs.
template <int RG>
__device__ __forceinline__ void gram_row_residual(const IterArgs &a, const BlockDesc &B, int r,
                                                  const double *__restrict__ y, int64_t ld,
                                                  int k0, uint32_t mask, double (&acc)[RG]) {
  const int sl = B.slice0 + (r >> 5), l = r & 31;
  const int64_t o = a.soff[sl];
  const int wd = (int)((a.soff[sl + 1] - o) >> 5);
  const double *sv = a.sval + o + l;
  const int16_t *sc = a.scol + o + l;
  if (mask == (RG == 32 ? 0xffffffffu : (1u << RG) - 1u) && (ld & 1) == 0) {
    for (int kk = 0; kk < wd; ++kk) {
      const double gv = sv[32 * kk];
      const double2 *yc = reinterpret_cast<const double2 *>(y + (B.row0 + sc[32 * kk]) * ld + k0);
#pragma unroll
      for (int h = 0; h < RG / 2; ++h) {
        const double2 t = yc[h];
        acc[2 * h] = fma(-gv, t.x, acc[2 * h]);
        acc[2 * h + 1] = fma(-gv, t.y, acc[2 * h + 1]);
      }
    }
  } else {
    for (int kk = 0; kk < wd; ++kk) {
      const double gv = sv[32 * kk];
      const double *yc = y + (B.row0 + sc[32 * kk]) * ld + k0;
#pragma unroll
      for (int g = 0; g < RG; ++g)
        if ((mask >> g) & 1u) acc[g] = fma(-gv, yc[g], acc[g]);
    }
  }
}

int proj_smem_bytes(int max_mp, int slots, int slot_bytes, int wbytes);
cudaError_t set_proj_smem_attr(int bytes);
// watchdog self-test: a bounded wait on an mbarrier nothing completes; sets bit 8 of *err
void launch_wait_selftest(uint64_t limit_ns, int32_t *err, cudaStream_t s);
// FP64 FMA throughput probe on every SM: returns the device milliseconds of `iters` rounds of
// 8 FMA chains per thread and writes the number of FMAs to *fmas
double launch_dfma_probe(int iters, double *sink, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                         int64_t *fmas);
// proj_mr_tc.cu: groups of 16 right-hand sides of FP32 blocks on the tensor cores
int proj_mr_tc_max_tiles();
size_t tile_map_bytes();
bool make_tile_map(void *map, const float *base, int64_t elems);
cudaError_t set_proj_mr_tc_smem_attr();
void launch_proj_mr_tc(const IterArgs &a, const double *u, double *y, int check_lane,
                       cudaStream_t s);
// proj_mr.cu: groups of rg right-hand sides share every factor tile read
int proj_mr_smem_bytes(int max_mp, int rg, int slots, int slot_bytes, int wbytes);
cudaError_t set_proj_mr_smem_attr(int rg, int bytes);
void launch_proj_mr(const IterArgs &a, const double *u, double *y, int check_lane,
                    cudaStream_t s);
void launch_rhs_scale(const IterArgs &a, const double *Fin, const int32_t *perm, cudaStream_t s);
void launch_spmv_plain(const IterArgs &a, const double *v, double *out, cudaStream_t s);
void launch_proj(const IterArgs &a, const double *u, double *y, int check_lane, cudaStream_t s);
void launch_spmv_t(const IterArgs &a, const double *y, double *out, cudaStream_t s);
void launch_cg_init(const IterArgs &a, cudaStream_t s);
// one CG iteration; e0 / e1 (may be null) are recorded around the projection launch
void launch_iteration(const IterArgs &a, cudaStream_t s, cudaEvent_t e0 = nullptr,
                      cudaEvent_t e1 = nullptr);
// one sweep of Algorithm 1: x += omega * sum_i A_i^+ (f_i - A_i x) (4 launches)
void launch_cim_sweep(const IterArgs &a, double omega, cudaStream_t s);
void launch_final_stats(const IterArgs &a, const double *Fin, const double *rowabs, double *out,
                        cudaStream_t s);
void launch_row_abs(const int64_t *rp, const int32_t *ci, const double *va, const double *d,
                    const double *cs, int64_t N, double *rowabs, cudaStream_t s);
// x (N x nrhs, [column][rhs]) /= cs per column: the column-scaled iterate back to x
void launch_unscale_cols(double *x, const double *cs, int64_t N, int32_t nrhs, cudaStream_t s);

}  // namespace cimmino
