// Batched Cholesky G_i = L_i L_i^T of the Gram blocks in FP64, in place on the tiled
// factor layout (tile rows J0(I)..I, T x T row-major tiles), right-looking over tile
// columns K:
//   1. factor the diagonal tile (in shared memory, 16 x 16 sub-blocks), record the pivots;
//   2. invert L_KK (kept in dinv for the triangular solves);
//   3. L_IK = G_IK * inv(L_KK)^T for the stored tiles below the diagonal;
//   4. G_IJ -= L_IK * L_JK^T for K < J <= I (only tiles inside the envelope exist,
//      and the fill of a Cholesky factor never leaves the envelope of G).
// Once row K is final (after step 2 of step K), its off-diagonal tiles are replaced by
// N_KJ = inv(L_KK) L_KJ, i.e. the factor is stored as L = diag(L_II) (I + N): the
// diagonal tiles keep L_II and dinv keeps inv(L_II).  The N transform runs afterwards in a
// kernel of its own (every tile independent).
// Pivot monitoring: min_j of the pivots L_jj^2 (G_jj = 1 after the unit row
// scaling) and a failure flag for a non-positive or non-finite pivot; a failed
// pivot is replaced by 1 so that the block finishes without NaNs.
//
// GB300's FP64 pipe bounds this kernel: each SM sub-partition issues about one FP64 warp
// instruction every 76 cycles (1.06 TFLOP/s over the GPU).  So every tile product is split
// into 16 x 16 output units, one warp per unit, balanced over the four sub-partitions, and
// the work that is zero by structure is skipped: the symmetric update of a diagonal tile
// computes its 36 lower 8 x 8 units only, and the products with the triangular inv(L_KK) run
// in 32 x 4 strips whose k loop ends where the triangle does (k <= column for G inv^T,
// k <= row for inv L).  The
// factorisation of a diagonal tile is a serial pivot chain on one sub-partition; with
// look-ahead (step 1 of K+1 on warps 0-3 beside step 4 of K on warps 4-7) the update fills
// the other sub-partitions meanwhile.
// Scheduling: one CTA per SM (shared memory keeps the others off) walks a list of blocks
// that the host packs from the blocks' tile counts; a block that would set the time alone
// is shared by two CTAs of a cooperative launch, which meet at bounded pair barriers.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace cimmino {

namespace {

constexpr int T = kTile;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int LD = T + 2;   // k-major operand rows (doubles): 16-byte aligned, staggered banks
constexpr int LDS = T + 1;  // padded row-major diagonal tile

__device__ __forceinline__ double *tile_ptr(double *fac, const TileRow &tr, int J) {
  return fac + tr.off + (int64_t)(J - tr.j0) * T * T;
}

// Global reads of factor tiles.  CG: through L2 only (ld.global.cg), for tiles that the other
// CTA of a split block writes (this SM's L1 may hold an older copy).
template <bool CG>
__device__ __forceinline__ double ldg(const double *p) {
  if (CG) return __ldcg(p);
  return *p;
}
template <bool CG>
__device__ __forceinline__ double2 ldg2(const double *p) {
  if (CG) return __ldcg(reinterpret_cast<const double2 *>(p));
  return *reinterpret_cast<const double2 *>(p);
}

// Load a row-major global tile into k-major shared storage At[k][r] = tile(r, k).
template <bool CG = false>
__device__ __forceinline__ void load_kmajor(const double *g, double *At) {
  for (int e = threadIdx.x; e < T * T; e += kThreads) {
    const int r = e / T, k = e % T;
    At[k * LD + r] = ldg<CG>(g + e);
  }
}
// Load a row-major global tile into row-major shared storage Bt[k][c] = tile(k, c).
__device__ __forceinline__ void load_rowmajor(const double *__restrict__ g, double *Bt) {
  for (int e = threadIdx.x; e < T * T / 2; e += kThreads) {
    const int k = e / (T / 2), c = 2 * (e % (T / 2));
    *reinterpret_cast<double2 *>(Bt + k * LD + c) = *reinterpret_cast<const double2 *>(g + k * T + c);
  }
}

// Output unit (R, C) of a 16 x 16 grid of a tile: lane (lr, lc) = (lane / 4, lane % 4) owns
// rows 16R + 2lr, +1 and columns 16C + 4lc .. +3.  acc = sum_{k < kend} At[k][r] Bt[k][c].
__device__ __forceinline__ void unit_product(const double *At, const double *Bt, int R, int C,
                                             int kend, double (&acc)[2][4]) {
  const int lane = threadIdx.x & 31, lr = lane >> 2, lc = lane & 3;
  const double *a = At + 16 * R + 2 * lr;
  const double *b = Bt + 16 * C + 4 * lc;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
#pragma unroll 4
  for (int k = 0; k < kend; ++k) {
    const double2 av = *reinterpret_cast<const double2 *>(a + k * LD);
    const double2 b0 = *reinterpret_cast<const double2 *>(b + k * LD);
    const double2 b1 = *reinterpret_cast<const double2 *>(b + k * LD + 2);
    const double ar[2] = {av.x, av.y}, br[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(ar[i], br[j], acc[i][j]);
  }
}

// Symmetric update of a diagonal tile, out -= At^T Bt on its lower triangle, in the 36 lower
// 8 x 8 units (R >= C; 16 x 16 units would leave 10 units to 8 or 4 warps, and compute the
// upper halves of their diagonal units): warp wl of nw takes units wl, wl + nw, ..., the same
// 9 units per SM sub-partition for nw = 8 and nw = 4.  Lane (lr, lc) = (lane / 4, lane % 4)
// owns row 8R + lr, columns 8C + 2lc, +1.  The upper parts of the diagonal units are written
// too (the upper triangle of a diagonal tile is never read).
template <bool CG = false>
__device__ __forceinline__ void sym_update8(const double *At, const double *Bt, double *out,
                                            int wl, int nw) {
  const int lane = threadIdx.x & 31, lr = lane >> 2, lc = lane & 3;
#pragma unroll 1
  for (int u = wl; u < 36; u += nw) {
    int R = 0;
    while ((R + 1) * (R + 2) / 2 <= u) ++R;
    const int C = u - R * (R + 1) / 2;
    const double *a = At + 8 * R + lr;
    const double *b = Bt + 8 * C + 2 * lc;
    double a0 = 0.0, a1 = 0.0;
#pragma unroll 8
    for (int k = 0; k < T; ++k) {
      const double x = a[k * LD];
      const double2 y = *reinterpret_cast<const double2 *>(b + k * LD);
      a0 = fma(x, y.x, a0);
      a1 = fma(x, y.y, a1);
    }
    double *q = out + (8 * R + lr) * T + 8 * C + 2 * lc;
    const double2 old = ldg2<CG>(q);
    *reinterpret_cast<double2 *>(q) = make_double2(old.x - a0, old.y - a1);
  }
}

// Products with a triangular factor in 32 x 4 strips, one warp each, so that the k bound is
// the same for the whole warp and follows the triangle to within 4 (16 x 16 units stop only at
// the unit's last column: 15% more FP64 instructions).
//   COLS (triangle in the columns of Bt, Bt[k][c] = 0 for k > c, the solves G inv(L)^T):
//     out(32h + lane, 4g + j) = sum_{k < 4g+4} At[k][32h + lane] Bt[k][4g + j], j < 4;
//   ROWS (triangle in the rows of At, At[k][r] = 0 for k > r, the transform inv(L) L_KJ):
//     out(4g + i, 32h + lane) = sum_{k < 4g+4} At[k][4g + i] Bt[k][32h + lane], i < 4.
// Strip (g, h) costs 4g + 4 k steps: warp w takes g = w and g = 15 - w for both h, the same
// 136 k steps for every warp and SM sub-partition.  The result is written to the row-major
// global tile out.
template <bool COLS>
__device__ __forceinline__ void tri_strips(const double *At, const double *Bt, double *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
  for (int v = 0; v < 4; ++v) {
    const int g = v < 2 ? warp : 15 - warp, h = v & 1;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int kend = 4 * g + 4;
#pragma unroll 4
    for (int k = 0; k < kend; ++k) {
      if (COLS) {
        const double a = At[k * LD + 32 * h + lane];
        const double2 b0 = *reinterpret_cast<const double2 *>(Bt + k * LD + 4 * g);
        const double2 b1 = *reinterpret_cast<const double2 *>(Bt + k * LD + 4 * g + 2);
        acc[0] = fma(a, b0.x, acc[0]);
        acc[1] = fma(a, b0.y, acc[1]);
        acc[2] = fma(a, b1.x, acc[2]);
        acc[3] = fma(a, b1.y, acc[3]);
      } else {
        const double2 a0 = *reinterpret_cast<const double2 *>(At + k * LD + 4 * g);
        const double2 a1 = *reinterpret_cast<const double2 *>(At + k * LD + 4 * g + 2);
        const double b = Bt[k * LD + 32 * h + lane];
        acc[0] = fma(a0.x, b, acc[0]);
        acc[1] = fma(a0.y, b, acc[1]);
        acc[2] = fma(a1.x, b, acc[2]);
        acc[3] = fma(a1.y, b, acc[3]);
      }
    }
    if (COLS) {
      double2 *o = reinterpret_cast<double2 *>(out + (32 * h + lane) * T + 4 * g);
      o[0] = make_double2(acc[0], acc[1]);
      o[1] = make_double2(acc[2], acc[3]);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) out[(4 * g + i) * T + 32 * h + lane] = acc[i];
    }
  }
}

// out(r, c) = acc (mode 0) or out(r, c) -= acc (mode 1) for the lane's elements of unit (R, C)
// of a row-major global tile.
template <bool CG = false>
__device__ __forceinline__ void unit_store(double *out, int R, int C, const double (&acc)[2][4],
                                           bool subtract) {
  const int lane = threadIdx.x & 31, lr = lane >> 2, lc = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    double *q = out + (16 * R + 2 * lr + i) * T + 16 * C + 4 * lc;
    double2 *p = reinterpret_cast<double2 *>(q);
    if (subtract) {
      const double2 x0 = ldg2<CG>(q), x1 = ldg2<CG>(q + 2);
      p[0] = make_double2(x0.x - acc[i][0], x0.y - acc[i][1]);
      p[1] = make_double2(x1.x - acc[i][2], x1.y - acc[i][3]);
    } else {
      p[0] = make_double2(acc[i][0], acc[i][1]);
      p[1] = make_double2(acc[i][2], acc[i][3]);
    }
  }
}

// Barrier of a group of NT threads: the whole CTA, or warps 0-3 (ID 1) / 4-7 (ID 2).
template <int ID, int NT>
__device__ __forceinline__ void group_sync() {
  if (NT == kThreads)
    __syncthreads();
  else
    asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(NT) : "memory");
}

// Cholesky L L^T of the 64 x 64 SPD tile in S (lower part read, L written over it) and inv(L)
// into the lower part of Di, by the first NT threads of the CTA (all of them, or warps 0-3
// with barrier 1), in 16 x 16 sub-blocks so that the 64 pivots
// take 12 barriers instead of two each:
//   block column k: warp 0 factors the diagonal sub-block (lane r holds row r in registers; the
//   columns of L reach the other rows by shuffles), the rows below solve against it (a thread
//   per row), and the trailing lower triangle, folded into a rectangle (rows p and n-1-p share
//   a line of n+1 entries), takes the rank-16 update;
//   inverse: warp k inverts diagonal sub-block k (a lane per column, in registers), and the
//   off-diagonal sub-blocks follow by distance d = i - k: Di_ik = -Di_ii sum_{k<=m<i} L_im Di_mk.
// Each FP64 operation on the pivot chain waits tens of cycles on GB300's narrow FP64 pipe, so a
// pivot costs one reciprocal square root (L_jj = d rsqrt(d), 1 / L_jj = rsqrt(d)), its chain
// stays in registers, and the lanes stay converged (selects instead of branches).  Entries
// above the diagonal of S are never read; Di's are zero inside the diagonal sub-blocks and
// unset elsewhere.  *pmin receives the smallest pivot of the first `rows` rows; a pivot that is
// not positive and finite sets *fail and is replaced by 1.  Tmp: 3 x 256 doubles.
template <int NT>
__device__ __noinline__ void diag_factor64(double *S, double *Di, double *Tmp, int rows,
                                           double *pmin, int *fail) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  double *rcp = Tmp;  // 1 / L_jj (Tmp is free until the off-diagonal inverse)
  for (int k = 0; k < 4; ++k) {
    const int b0 = 16 * k;
    if (warp == 0) {
      const int r = lane & 15;
      double a[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) a[c] = S[(b0 + r) * LDS + b0 + c];
      double pm = INFINITY;
      bool bad = false;
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int j = b0 + jj;
        double d = __shfl_sync(0xffffffffu, a[jj], jj);
        if (j < rows) pm = fmin(pm, d);
        if (!(d > 0.0) || !isfinite(d)) {
          bad = true;
          d = 1.0;
        }
        const double rc = rsqrt(d), l = d * rc;
        if (lane == jj) rcp[j] = rc;
        a[jj] = r == jj ? l : (r > jj ? a[jj] * rc : a[jj]);
        double lc[16];
#pragma unroll
        for (int c = jj + 1; c < 16; ++c) lc[c] = __shfl_sync(0xffffffffu, a[jj], c);
#pragma unroll
        for (int c = jj + 1; c < 16; ++c) a[c] = r >= c ? fma(-a[jj], lc[c], a[c]) : a[c];
      }
      if (lane < 16) {
#pragma unroll
        for (int c = 0; c < 16; ++c) S[(b0 + r) * LDS + b0 + c] = a[c];
      }
      if (lane == 0) {
        if (pm < INFINITY) *pmin = fmin(*pmin, pm);
        if (bad) *fail = 1;
      }
    }
    group_sync<1, NT>();
    if (k == 3) break;
    // rows below: L_ic = S_ic L_cc^-T, forward substitution along the row, a thread per row
    const int i = b0 + 16 + t;
    if (i < T) {
      double x[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        double v = S[i * LDS + b0 + c];
#pragma unroll
        for (int m = 0; m < c; ++m) v = fma(-x[m], S[(b0 + c) * LDS + b0 + m], v);
        x[c] = v * rcp[b0 + c];
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) S[i * LDS + b0 + c] = x[c];
    }
    group_sync<1, NT>();
    // trailing lower triangle: S_ic -= sum_m L_im L_cm over the block column
    const int n = T - b0 - 16, w = n + 1;
    for (int e = t; e < (n / 2) * w; e += NT) {
      const int p = e / w, q = e % w;
      const int ii = b0 + 16 + (q <= p ? p : n - 1 - p);
      const int c = b0 + 16 + (q <= p ? q : q - p - 1);
      double v = S[ii * LDS + c];
#pragma unroll
      for (int m = 0; m < 16; ++m) v = fma(-S[ii * LDS + b0 + m], S[c * LDS + b0 + m], v);
      S[ii * LDS + c] = v;
    }
    group_sync<1, NT>();
  }
  // inverse of every diagonal sub-block: warp k, lane c < 16 owns column c (entries above the
  // diagonal are zero, so the sums may start at m = 0)
  if (warp < 4) {
    const int b0 = 16 * warp, c = lane & 15;
    double col[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const double ri = rcp[b0 + i];
      double v = 0.0;
#pragma unroll
      for (int m = 0; m < i; ++m) v = fma(-S[(b0 + i) * LDS + b0 + m], col[m], v);
      col[i] = i < c ? 0.0 : (i == c ? ri : v * ri);
    }
    if (lane < 16) {
#pragma unroll
      for (int i = 0; i < 16; ++i) Di[(b0 + i) * LDS + b0 + c] = col[i];
    }
  }
  group_sync<1, NT>();
  for (int d = 1; d < 4; ++d) {
    const int np = 4 - d;  // sub-block pairs (i, k = i - d), i = d..3
    // Tmp_p = sum_{k <= m < i} L_im Di_mk
    for (int e = t; e < np * 256; e += NT) {
      const int p = e >> 8, r = (e >> 4) & 15, c = e & 15;
      const int bi = d + p, bk = p;
      double v = 0.0;
      for (int m = 16 * bk; m < 16 * bi; ++m)
        v = fma(S[(16 * bi + r) * LDS + m], Di[m * LDS + 16 * bk + c], v);
      Tmp[e] = v;
    }
    group_sync<1, NT>();
    // Di_ik = -Di_ii Tmp_p
    for (int e = t; e < np * 256; e += NT) {
      const int p = e >> 8, r = (e >> 4) & 15, c = e & 15;
      const int bi = d + p, bk = p;
      double v = 0.0;
#pragma unroll
      for (int m = 0; m < 16; ++m)
        v = fma(Di[(16 * bi + r) * LDS + 16 * bi + m], Tmp[(p << 8) + m * 16 + c], v);
      Di[(16 * bi + r) * LDS + 16 * bk + c] = -v;
    }
    group_sync<1, NT>();
  }
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr uint64_t kPairWaitNs = 2000000000ull;  // a pair wait gives up after ~2 s
constexpr uint32_t kPairSpins = 1u << 26;         // ... or after this many polls

// Barrier of the two CTAs that share a split block: each publishes its epoch in flag[part]
// and waits, bounded, until flag[1 - part] has reached it.  The fences order the tile writes
// before the barrier ahead of the other CTA's reads after it, which go to L2 (CG loads).
// Returns false (and sets `bit` in *err) when the wait ran out.
__device__ bool pair_sync(int32_t *flag, int part, int32_t epoch, int32_t *err, int *s_ok,
                          uint64_t limit_ns = kPairWaitNs, int32_t bit = 1) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(flag + part, epoch);
    int ok = 1;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0;; ++i) {
      int32_t v;
      asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(flag + 1 - part) : "memory");
      if (v >= epoch) break;
      if (i >= kPairSpins || global_ns() - t0 > limit_ns) {
        atomicOr(err, bit);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Right-looking Cholesky of one Gram block (the steps in the file header) shared by two CTAs
// (part 0 and 1) that meet at pair barriers three times per tile column: part 0 factors the
// diagonal tile; the triangular solves alternate between the parts; the update rows go to the
// part with less update work so far (largest rows first).  Tiles the other part writes are
// read through L2 (CG loads).
__device__ __forceinline__ void factor_block_split(const BlockDesc &B, int b, int part, int32_t *flag,
                                             const TileRow *__restrict__ trow,
                                             double *__restrict__ fac, double *__restrict__ dinv,
                                             double *__restrict__ pivmin,
                                             int32_t *__restrict__ pivfail, int32_t *err,
                                             double *At, double *Bt, double *Tmp,
                                             TileRow *s_tr, unsigned char *s_own, double &s_pmin,
                                             int &s_fail, int &s_ok) {
  double *S = At;   // [T][LDS], diagonal phase only
  double *Di = Bt;  // [T][LDS], diagonal phase only
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int I = tid; I < B.nt; I += kThreads) s_tr[I] = trow[B.trow0 + I];
  const TileRow *tr = s_tr;
  if (tid == 0) {
    s_pmin = 1e300;
    s_fail = 0;
  }
  __syncthreads();
  int32_t epoch = 0;
  for (int K = 0; K < B.nt; ++K) {
    const TileRow TK = tr[K];
    double *gKK = tile_ptr(fac, TK, K);
    double *dK = dinv + B.dinv_off + (int64_t)K * T * T;
    if (part == 0) {
      // ---- 1-2. factor the diagonal tile and invert it, in shared memory
      for (int e = tid; e < T * T; e += kThreads) S[(e / T) * LDS + (e % T)] = ldg<true>(gKK + e);
      __syncthreads();
      diag_factor64<kThreads>(S, Di, Tmp, B.m - K * T, &s_pmin, &s_fail);
      // write L_KK (upper part zeroed) and inv(L_KK)
      for (int e = tid; e < T * T; e += kThreads) {
        const int r = e / T, c = e % T;
        gKK[e] = c <= r ? S[r * LDS + c] : 0.0;
        dK[e] = c <= r ? Di[r * LDS + c] : 0.0;
      }
    }
    if (!pair_sync(flag, part, ++epoch, err, &s_ok)) break;
    // Bt[k][c] = inv(L_KK)(c, k) for the triangular solves below (upper triangular); read back
    // from dinv
    load_kmajor<true>(dK, Bt);
    __syncthreads();
    // ---- 3. L_IK = G_IK * Di^T for every stored tile below the diagonal
    int q = 0;
    for (int I = K + 1; I < B.nt; ++I) {
      const TileRow TI = tr[I];
      if (TI.j0 > K) continue;
      if ((q++ & 1) != part) continue;
      double *gIK = tile_ptr(fac, TI, K);
      load_kmajor<true>(gIK, At);
      __syncthreads();
      tri_strips<true>(At, Bt, gIK);  // inv(L_KK)^T is upper triangular
      __syncthreads();
    }
    if (!pair_sync(flag, part, ++epoch, err, &s_ok)) break;
    // rows of the update: row I costs its tiles (K, I) inside the envelope (3/4 for the
    // symmetric diagonal one); the larger rows first, each to the part with less so far
    if (tid == 0) {
      int w[2] = {0, 0};
      int act = 0;  // envelope rows in K+1..I
      for (int I = K + 1; I < B.nt; ++I) act += tr[I].j0 <= K;
      for (int I = B.nt - 1; I > K; --I) {
        if (tr[I].j0 > K) continue;
        const int cost = 4 * act - 1;  // (act - 1) full tiles + 3/4, in quarters
        const int pick = w[1] < w[0] ? 1 : 0;
        s_own[I] = (unsigned char)pick;
        w[pick] += cost;
        --act;
      }
    }
    __syncthreads();
    // ---- 4. trailing update G_IJ -= L_IK L_JK^T; a diagonal tile (J = I) is symmetric and
    // only its lower units are updated (the upper triangle of G_II is never read)
    for (int I = K + 1; I < B.nt; ++I) {
      const TileRow TI = tr[I];
      if (TI.j0 > K) continue;
      if (s_own[I] != part) continue;
      load_kmajor<true>(tile_ptr(fac, TI, K), At);
      for (int J = K + 1; J <= I; ++J) {
        const TileRow TJ = tr[J];
        if (TJ.j0 > K) continue;
        __syncthreads();  // previous use of Bt finished
        load_kmajor<true>(tile_ptr(fac, TJ, K), Bt);
        __syncthreads();
        double *gIJ = tile_ptr(fac, TI, J);
        if (J < I) {
          for (int u = warp; u < 16; u += kWarps) {
            const int R = u >> 2, C = u & 3;
            double acc[2][4];
            unit_product(At, Bt, R, C, T, acc);
            unit_store<true>(gIJ, R, C, acc, true);
          }
        } else {
          sym_update8<true>(At, Bt, gIJ, warp, kWarps);
        }
      }
      __syncthreads();
    }
    if (!pair_sync(flag, part, ++epoch, err, &s_ok)) break;
  }
  if (tid == 0 && part == 0) {
    pivmin[b] = s_pmin;
    pivfail[b] = s_fail;
  }
  __syncthreads();  // the shared tables are reused by the CTA's next block
}

// Watchdog self-test of the pair wait: part 0 of a pair whose partner never arrives (flag[1]
// stays 0) must give up after limit_ns and set bit 16 of the error word.
__global__ void __launch_bounds__(kThreads) k_pair_selftest(uint64_t limit_ns, int32_t *flag,
                                                            int32_t *err) {
  __shared__ int s_ok;
  pair_sync(flag, 0, 1, err, &s_ok, limit_ns, 16);
}

// The diagonal tile K factored and inverted by warps 0-3 (barrier 1) in their own shared
// memory S, Di, Tmp; L_KK and inv(L_KK) are written to fac and dinv.
__device__ __forceinline__ void factor_diag_group(const BlockDesc &B, const TileRow *tr, int K,
                                                  double *fac, double *dinv, double *S,
                                                  double *Di, double *Tmp, double *pmin,
                                                  int *fail) {
  const int t = threadIdx.x;
  double *gKK = tile_ptr(fac, tr[K], K);
  for (int e = t; e < T * T; e += 128) S[(e / T) * LDS + (e % T)] = gKK[e];
  group_sync<1, 128>();
  diag_factor64<128>(S, Di, Tmp, B.m - K * T, pmin, fail);
  double *dK = dinv + B.dinv_off + (int64_t)K * T * T;
  for (int e = t; e < T * T; e += 128) {
    const int r = e / T, c = e % T;
    gKK[e] = c <= r ? S[r * LDS + c] : 0.0;
    dK[e] = c <= r ? Di[r * LDS + c] : 0.0;
  }
}

// Right-looking Cholesky of one Gram block by one CTA with look-ahead.  Step K: all 8 warps
// solve the tiles (I, K) and update column K+1 (the tiles (I, K+1)); then warps 0-3 factor
// the diagonal tile K+1 while warps 4-7 update the rest of the trailing matrix (columns K+2 and
// on).  The factorisation of a diagonal tile is a serial pivot chain that keeps one SM
// sub-partition busy at a time; the update warps fill the other three meanwhile.
__device__ __forceinline__ void factor_block_la(const BlockDesc &B, int b,
                                                const TileRow *__restrict__ trow,
                                                double *__restrict__ fac,
                                                double *__restrict__ dinv,
                                                double *__restrict__ pivmin,
                                                int32_t *__restrict__ pivfail, double *At,
                                                double *Bt, double *Sf, double *Dif,
                                                double *Tmpf, TileRow *s_tr, double &s_pmin,
                                                int &s_fail) {
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int I = tid; I < B.nt; I += kThreads) s_tr[I] = trow[B.trow0 + I];
  if (tid == 0) {
    s_pmin = 1e300;
    s_fail = 0;
  }
  __syncthreads();
  const TileRow *tr = s_tr;
  if (warp < 4) factor_diag_group(B, tr, 0, fac, dinv, Sf, Dif, Tmpf, &s_pmin, &s_fail);
  __syncthreads();
  for (int K = 0; K < B.nt; ++K) {
    // Bt[k][c] = inv(L_KK)(c, k) for the triangular solves (upper triangular)
    load_kmajor(dinv + B.dinv_off + (int64_t)K * T * T, Bt);
    __syncthreads();
    // ---- 3. L_IK = G_IK * inv(L_KK)^T for every stored tile below the diagonal
    for (int I = K + 1; I < B.nt; ++I) {
      const TileRow TI = tr[I];
      if (TI.j0 > K) continue;
      double *gIK = tile_ptr(fac, TI, K);
      load_kmajor(gIK, At);
      __syncthreads();
      tri_strips<true>(At, Bt, gIK);  // inv(L_KK)^T is upper triangular
      __syncthreads();
    }
    // ---- 4a. column K+1 of the trailing update, G_{I,K+1} -= L_IK L_{K+1,K}^T (all warps)
    if (K + 1 < B.nt && tr[K + 1].j0 <= K) {
      load_kmajor(tile_ptr(fac, tr[K + 1], K), Bt);
      for (int I = K + 1; I < B.nt; ++I) {
        const TileRow TI = tr[I];
        if (TI.j0 > K) continue;
        load_kmajor(tile_ptr(fac, TI, K), At);
        __syncthreads();
        double *g = tile_ptr(fac, TI, K + 1);
        if (I > K + 1) {
          for (int u = warp; u < 16; u += kWarps) {
            const int R = u >> 2, C = u & 3;
            double acc[2][4];
            unit_product(At, Bt, R, C, T, acc);
            unit_store(g, R, C, acc, true);
          }
        } else {
          sym_update8(At, Bt, g, warp, kWarps);
        }
        __syncthreads();
      }
    }
    if (warp < 4) {
      // ---- 1-2 of step K+1: the diagonal tile K+1 (updated by every step up to K)
      if (K + 1 < B.nt) factor_diag_group(B, tr, K + 1, fac, dinv, Sf, Dif, Tmpf, &s_pmin, &s_fail);
    } else {
      // ---- 4b. the rest of the trailing update, G_IJ -= L_IK L_JK^T for K+2 <= J <= I, by
      // warps 4-7 (barrier 2); a diagonal tile (J = I) takes its lower units only
      const int tu = tid - 128, wl = warp - 4;
      for (int I = K + 2; I < B.nt; ++I) {
        const TileRow TI = tr[I];
        if (TI.j0 > K) continue;
        const double *gIK = tile_ptr(fac, TI, K);
        for (int e = tu; e < T * T; e += 128) At[(e % T) * LD + e / T] = gIK[e];
        for (int J = K + 2; J <= I; ++J) {
          const TileRow TJ = tr[J];
          if (TJ.j0 > K) continue;
          group_sync<2, 128>();  // previous use of Bt finished
          const double *gJK = tile_ptr(fac, TJ, K);
          for (int e = tu; e < T * T; e += 128) Bt[(e % T) * LD + e / T] = gJK[e];
          group_sync<2, 128>();
          double *gIJ = tile_ptr(fac, TI, J);
          if (J < I) {
            for (int u = wl; u < 16; u += 4) {
              const int R = u >> 2, C = u & 3;
              double acc[2][4];
              unit_product(At, Bt, R, C, T, acc);
              unit_store(gIJ, R, C, acc, true);
            }
          } else {
            sym_update8(At, Bt, gIJ, wl, 4);
          }
        }
        group_sync<2, 128>();  // At free for the next row
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    pivmin[b] = s_pmin;
    pivfail[b] = s_fail;
  }
  __syncthreads();  // the shared tables are reused by the CTA's next block
}

// One CTA per SM walks its list of blocks items[cta_ptr[c] .. cta_ptr[c + 1]) (a static
// schedule packed on the host from the blocks' measured tile costs); an item with nparts = 2
// is half of a split block, first in the lists of both CTAs that share it.
__global__ void __launch_bounds__(kThreads, 1)
    k_cholesky(const BlockDesc *__restrict__ blk, const CholItem *__restrict__ items,
               const int32_t *__restrict__ cta_ptr, const TileRow *__restrict__ trow,
               double *__restrict__ fac, double *__restrict__ dinv, double *__restrict__ pivmin,
               int32_t *__restrict__ pivfail, int32_t *__restrict__ pair_flags,
               int32_t *__restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *At = reinterpret_cast<double *>(smem_raw);  // [T][LD]
  double *Bt = At + T * LD;                            // [T][LD]
  double *Sf = Bt + T * LD;                            // [T][LDS], warps 0-3's diagonal tile
  double *Dif = Sf + T * LDS;                          // [T][LDS]
  double *Tmpf = Dif + T * LDS;                        // [3 * 256]
  __shared__ double s_pmin;
  __shared__ int s_fail, s_ok;
  __shared__ TileRow s_tr[kMaxBlockRows / T];  // the block's tile-row table
  __shared__ unsigned char s_own[kMaxBlockRows / T];
  for (int32_t i = cta_ptr[blockIdx.x]; i < cta_ptr[blockIdx.x + 1]; ++i) {
    const CholItem it = items[i];
    const BlockDesc B = blk[it.b];
    if (it.nparts == 2)
      factor_block_split(B, it.b, it.part, pair_flags + 2 * it.slot, trow, fac, dinv, pivmin,
                         pivfail, err, At, Bt, Tmpf, s_tr, s_own, s_pmin, s_fail, s_ok);
    else
      factor_block_la(B, it.b, trow, fac, dinv, pivmin, pivfail, At, Bt, Sf, Dif, Tmpf, s_tr,
                      s_pmin, s_fail);
  }
}

// Transposed copy of a factor for the backward solves: upper tile row I holds
// NT_IJ = N_JI^T for J = I+1..J1(I) (J1(I) = last tile row whose envelope reaches
// column I; tiles with J0(J) > I are zero), and dinvT_I = inv(L_II)^T.
template <typename W>
__device__ void transpose_block(const BlockDesc &B, const TileRow *__restrict__ tr,
                                const TileRow *__restrict__ trT, const W *__restrict__ fac,
                                const W *__restrict__ dinv, W *__restrict__ facT,
                                W *__restrict__ dinvT, W *sm) {
  constexpr int LDS = T + 1;
  auto tile_t = [&](const W *src, W *dst) {
    __syncthreads();
    for (int e = threadIdx.x; e < T * T; e += kThreads) sm[(e / T) * LDS + (e % T)] = src[e];
    __syncthreads();
    for (int e = threadIdx.x; e < T * T; e += kThreads) dst[e] = sm[(e % T) * LDS + (e / T)];
  };
  // tile row I of the transposed copy: one CTA per (block, tile row)
  const int I = blockIdx.y;
  if (I >= B.nt) return;
  tile_t(dinv + B.dinv_off + (int64_t)I * T * T, dinvT + B.dinv_off + (int64_t)I * T * T);
  const TileRow U = trT[I];
  for (int J = I + 1; J <= U.j0; ++J) {
    W *dst = facT + U.off + (int64_t)(J - I - 1) * T * T;
    const TileRow R = tr[J];
    if (R.j0 <= I) {
      tile_t(fac + R.off + (int64_t)(I - R.j0) * T * T, dst);
    } else {
      for (int e = threadIdx.x; e < T * T; e += kThreads) dst[e] = W(0);
    }
  }
}

// Packed copies of inv(L_II) (lower) and inv(L_II)^T (upper) for the single-vector solves
// of FP64 blocks:
// entry j of row pair p is (p, j) for j <= p and (63 - p, j - p - 1) for p < j <= 64 (lower),
// (p, p + j) for j <= 63 - p and (63 - p, j - 1) for 63 - p < j <= 64 (upper); the rest 0.
template <typename W>
__device__ void pack_block(const BlockDesc &B, const W *__restrict__ dinv,
                           const W *__restrict__ dinvT, W *__restrict__ P, W *__restrict__ PT) {
  const int64_t o = B.dinv_off, op = B.dinv_off / (T * T) * kPackTile;
  for (int64_t e = threadIdx.x; e < (int64_t)B.nt * kPackTile; e += kThreads) {
    const int I = (int)(e / kPackTile), q = (int)(e % kPackTile);
    const int p = q / kPackPair, j = q % kPackPair;
    const W *D = dinv + o + (int64_t)I * T * T;
    const W *DT = dinvT + o + (int64_t)I * T * T;
    W lv = W(0), uv = W(0);
    if (j <= p)
      lv = D[p * T + j];
    else if (j <= 64)
      lv = D[(63 - p) * T + (j - p - 1)];
    if (j <= 63 - p)
      uv = DT[p * T + p + j];
    else if (j <= 64)
      uv = DT[(63 - p) * T + (j - 1)];
    P[op + e] = lv;
    PT[op + e] = uv;
  }
}

// Block-packed copies for FP32 blocks: row pair p (b = p / 16) holds, for the lower tile,
// row p columns 0 .. 16 (b + 1) - 1 and then row 63 - p columns 0 .. 16 (4 - b) - 1; for
// the upper tile row p columns 16 b .. 63 and then row 63 - p columns 16 (3 - b) .. 63;
// 80 values (entries outside the triangle inside a diagonal sub-tile are zero), padded to
// kBPackPair.
__device__ void bpack_block(const BlockDesc &B, const float *__restrict__ dinv,
                            const float *__restrict__ dinvT, float *__restrict__ P,
                            float *__restrict__ PT) {
  const int64_t o = B.dinv_off, op = B.dinv_off / (T * T) * kBPackTile;
  for (int64_t e = threadIdx.x; e < (int64_t)B.nt * kBPackTile; e += kThreads) {
    const int I = (int)(e / kBPackTile), q = (int)(e % kBPackTile);
    const int p = q / kBPackPair, j = q % kBPackPair, b = p / 16;
    const float *D = dinv + o + (int64_t)I * T * T;
    const float *DT = dinvT + o + (int64_t)I * T * T;
    const int la = 16 * (b + 1), ua = 16 * (4 - b);  // entries of the pair's first row
    float lv = 0.f, uv = 0.f;
    if (j < la)
      lv = D[p * T + j];
    else if (j < 80)
      lv = D[(63 - p) * T + (j - la)];
    if (j < ua)
      uv = DT[p * T + 16 * b + j];
    else if (j < 80)
      uv = DT[(63 - p) * T + 16 * (3 - b) + (j - ua)];
    P[op + e] = lv;
    PT[op + e] = uv;
  }
}

__global__ void __launch_bounds__(kThreads)
    k_pack_diag(const BlockDesc *__restrict__ blk, FactorPtrs f) {
  const BlockDesc B = blk[blockIdx.x];
  if (B.prec64)
    pack_block<double>(B, f.dinv64, f.dinvT64, f.dinvP64, f.dinvTP64);
  else
    bpack_block(B, f.dinv32, f.dinvT32, f.dinvP32, f.dinvTP32);
}

__global__ void __launch_bounds__(kThreads)
    k_transpose_factor(const BlockDesc *__restrict__ blk, const TileRow *__restrict__ trow,
                       const TileRow *__restrict__ trowT, FactorPtrs f) {
  __shared__ double sm[T * (T + 1)];
  const BlockDesc B = blk[blockIdx.x];
  if (B.prec64)
    transpose_block<double>(B, trow + B.trow0, trowT + B.trow0, f.fac64, f.dinv64, f.facT64,
                            f.dinvT64, sm);
  else
    transpose_block<float>(B, trow + B.trow0, trowT + B.trow0, f.fac32, f.dinv32, f.facT32,
                           f.dinvT32, reinterpret_cast<float *>(sm));
}

// N_KJ = inv(L_KK) L_KJ in place for every off-diagonal tile of tile row K of the listed
// blocks (one CTA per block and tile row); inv(L_KK) is lower triangular, so the strips of
// rows 4g..4g+3 stop at k = 4g + 4.
__global__ void __launch_bounds__(kThreads)
    k_ntransform64(const BlockDesc *__restrict__ blk, const int32_t *__restrict__ blist,
                   const TileRow *__restrict__ trow, double *__restrict__ fac,
                   const double *__restrict__ dinv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *At = reinterpret_cast<double *>(smem_raw);  // At[k][r] = inv(L_KK)(r, k)
  double *Bt = At + T * LD;                            // Bt[k][c] = L_KJ(k, c)
  const BlockDesc B = blk[blist[blockIdx.x]];
  const int K = blockIdx.y;
  if (K >= B.nt) return;
  const TileRow TK = trow[B.trow0 + K];
  if (TK.j0 >= K) return;
  load_kmajor(dinv + B.dinv_off + (int64_t)K * T * T, At);
  for (int J = TK.j0; J < K; ++J) {
    double *g = tile_ptr(fac, TK, J);
    __syncthreads();
    load_rowmajor(g, Bt);
    __syncthreads();
    tri_strips<false>(At, Bt, g);  // inv(L_KK) is lower triangular
  }
}

constexpr int kCholSmem = (int)sizeof(double) * 2 * T * LD;      // operand tiles
// + the look-ahead group's diagonal tile, its inverse and scratch
constexpr int kCholSmemDiag = kCholSmem + (int)sizeof(double) * (2 * T * LDS + 3 * 256);
// dynamic shared memory of k_cholesky (one CTA per SM)
constexpr int kCholSmemLaunch = kCholSmemDiag;
static_assert(T * LDS <= T * LD, "diagonal scratch inside an operand tile");
static_assert(kCholSmemLaunch >= kCholSmemDiag, "launch reservation covers the tiles");
static_assert(kWarps == 8, "unit maps assume 8 warps");

}  // namespace

void launch_pair_selftest(uint64_t limit_ns, int32_t *flag, int32_t *err, cudaStream_t s) {
  k_pair_selftest<<<1, kThreads, 0, s>>>(limit_ns, flag, err);
}

int32_t cholesky_resident_ctas() {
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kCholSmemLaunch) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cholesky, kThreads,
                                                    kCholSmemLaunch) != cudaSuccess)
    return 0;
  return nsm * per_sm;
}

cudaError_t launch_cholesky(const BlockDesc *blk, const CholItem *items, const int32_t *cta_ptr,
                            int32_t ncta, bool cooperative, const TileRow *trow, double *fac,
                            double *dinv, double *pivmin, int32_t *pivfail, int32_t *pair_flags,
                            int32_t *err, cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
  cudaError_t e =
      cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, kCholSmemLaunch);
  if (e != cudaSuccess) return e;
  if (!cooperative) {
    k_cholesky<<<(unsigned)ncta, kThreads, kCholSmemLaunch, s>>>(blk, items, cta_ptr, trow, fac,
                                                                dinv, pivmin, pivfail, pair_flags,
                                                                err);
    return cudaGetLastError();
  }
  void *args[] = {(void *)&blk,    (void *)&items,   (void *)&cta_ptr,    (void *)&trow,
                  (void *)&fac,    (void *)&dinv,    (void *)&pivmin,     (void *)&pivfail,
                  (void *)&pair_flags, (void *)&err};
  return cudaLaunchCooperativeKernel((const void *)k_cholesky, dim3((unsigned)ncta),
                                     dim3(kThreads), args, (size_t)kCholSmemLaunch, s);
}

void launch_ntransform64(const BlockDesc *blk, const int32_t *blist, int32_t nlist,
                         const TileRow *trow, double *fac, const double *dinv, cudaStream_t s) {
  if (nlist <= 0) return;
  cudaFuncSetAttribute(k_ntransform64, cudaFuncAttributeMaxDynamicSharedMemorySize, kCholSmem);
  k_ntransform64<<<dim3((unsigned)nlist, kMaxBlockRows / T), kThreads, kCholSmem, s>>>(
      blk, blist, trow, fac, dinv);
}

void launch_transpose_factor(const BlockDesc *blk, int32_t nblk, const TileRow *trow,
                             const TileRow *trowT, const FactorPtrs &f, cudaStream_t s) {
  if (nblk > 0)
    k_transpose_factor<<<dim3((unsigned)nblk, kMaxBlockRows / T), kThreads, 0, s>>>(blk, trow,
                                                                                    trowT, f);
  if (nblk > 0) k_pack_diag<<<(unsigned)nblk, kThreads, 0, s>>>(blk, f);
}

}  // namespace cimmino
