// Batched Cholesky G_i = L_i L_i^T of the Gram blocks in FP64, in place on the tiled
// factor layout (tile rows J0(I)..I, T x T row-major tiles).  One CTA per block,
// right-looking over tile columns K:
//   1. factor the diagonal tile (unblocked, in shared memory), record the pivots;
//   2. invert L_KK (kept in dinv for the triangular solves);
//   3. L_IK = G_IK * inv(L_KK)^T for the stored tiles below the diagonal;
//   4. G_IJ -= L_IK * L_JK^T for K < J <= I (only tiles inside the envelope exist,
//      and the fill of a Cholesky factor never leaves the envelope of G).
// Once row K is final (after step 2 of step K), its off-diagonal tiles are replaced by
// N_KJ = inv(L_KK) L_KJ, i.e. the factor is stored as L = diag(L_II) (I + N): the
// diagonal tiles keep L_II and dinv keeps inv(L_II).
// Pivot monitoring: min_j of the pivots L_jj^2 (G_jj = 1 after the unit row
// scaling) and a failure flag for a non-positive or non-finite pivot; a failed
// pivot is replaced by 1 so that the block finishes without NaNs.
//
// GB300's FP64 pipe (about 2 FMA lanes per cycle per SM) bounds this kernel, so every
// tile product is split into 16 x 16 output units, one warp per unit, and the units skip
// the work that is zero by structure: the symmetric update of a diagonal tile computes
// its 10 lower units only, and products with the triangular inv(L_KK) stop the k loop
// where the triangle ends (k <= column for G inv^T, k <= row for inv L).  Work is then
// close to the algorithmic count.  The N transform of row K runs afterwards in a kernel of
// its own (every tile independent), and the diagonal scratch shares shared memory with the
// operand tiles.  One block per SM: on the 512-block random workload (n = 2^20) the
// factorisation took 79.9 ms with one, 87.3 ms with two and 99.7 ms with three blocks per
// SM, so the launch reserves enough shared memory to keep the others off the SM (the rest
// of the SM's 256 KB stays L1 for the tiles every product re-reads).
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

// Load a row-major global tile into k-major shared storage At[k][r] = tile(r, k).
__device__ __forceinline__ void load_kmajor(const double *__restrict__ g, double *At) {
  for (int e = threadIdx.x; e < T * T; e += kThreads) {
    const int r = e / T, k = e % T;
    At[k * LD + r] = g[e];
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

// The 10 lower units (R >= C) of a symmetric tile, in the order R = 0..3, C = 0..R.
__device__ __forceinline__ void lower_unit(int u, int &R, int &C) {
  R = u >= 6 ? 3 : u >= 3 ? 2 : u >= 1 ? 1 : 0;
  C = u - R * (R + 1) / 2;
}

// out(r, c) = acc (mode 0) or out(r, c) -= acc (mode 1) for the lane's elements of unit (R, C)
// of a row-major global tile.
__device__ __forceinline__ void unit_store(double *out, int R, int C, const double (&acc)[2][4],
                                           bool subtract) {
  const int lane = threadIdx.x & 31, lr = lane >> 2, lc = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    double2 *p = reinterpret_cast<double2 *>(out + (16 * R + 2 * lr + i) * T + 16 * C + 4 * lc);
    if (subtract) {
      const double2 x0 = p[0], x1 = p[1];
      p[0] = make_double2(x0.x - acc[i][0], x0.y - acc[i][1]);
      p[1] = make_double2(x1.x - acc[i][2], x1.y - acc[i][3]);
    } else {
      p[0] = make_double2(acc[i][0], acc[i][1]);
      p[1] = make_double2(acc[i][2], acc[i][3]);
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1)
    k_cholesky(const BlockDesc *__restrict__ blk, const int32_t *__restrict__ blist,
               const TileRow *__restrict__ trow, double *__restrict__ fac,
               double *__restrict__ dinv, double *__restrict__ pivmin,
               int32_t *__restrict__ pivfail) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *At = reinterpret_cast<double *>(smem_raw);  // [T][LD]
  double *Bt = At + T * LD;                            // [T][LD]
  double *S = At;                                      // [T][LDS], diagonal phase only
  double *Di = Bt;                                     // [T][LDS], diagonal phase only
  __shared__ double s_pmin;
  __shared__ int s_fail;
  __shared__ TileRow s_tr[kMaxBlockRows / T];  // the block's tile-row table
  __shared__ double s_rcp[T], s_d[T];            // pivots and their reciprocals

  const int b = blist[blockIdx.x];
  const BlockDesc B = blk[b];
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int I = tid; I < B.nt; I += kThreads) s_tr[I] = trow[B.trow0 + I];
  const TileRow *tr = s_tr;
  const int tr4 = tid / 16, tc4 = tid % 16;
  if (tid == 0) {
    s_pmin = 1e300;
    s_fail = 0;
  }
  __syncthreads();

  for (int K = 0; K < B.nt; ++K) {
    const TileRow TK = tr[K];
    double *gKK = tile_ptr(fac, TK, K);
    // ---- 1. diagonal tile, right-looking with the column scaling deferred: step j
    // subtracts S_ij S_kj / d_j from the trailing triangle (one barrier per column);
    // afterwards L_jj = sqrt(d_j) and L_ij = S_ij / sqrt(d_j)
    // Divisions and square roots run as long FP64 sequences on GB300's narrow FP64 pipe,
    // whose cost is per warp instruction: each reciprocal is computed by one warp only
    // (warp 0, lane 0) and shared, never by every warp.
    for (int e = tid; e < T * T; e += kThreads) S[(e / T) * LDS + (e % T)] = gKK[e];
    __syncthreads();
    for (int j = 0; j < T; ++j) {
      if (tid == 0) {
        double dj = S[j * LDS + j];
        if (K * T + j < B.m) s_pmin = fmin(s_pmin, dj);
        if (!(dj > 0.0) || !isfinite(dj)) {
          s_fail = 1;
          dj = 1.0;
        }
        s_rcp[j] = 1.0 / dj;
        s_d[j] = dj;
      }
      __syncthreads();
      const double inv = s_rcp[j];
      for (int i = j + 1 + tr4; i < T; i += 16) {
        const double t = S[i * LDS + j] * inv;
        for (int k = j + 1 + tc4; k <= i; k += 16) S[i * LDS + k] = fma(-t, S[k * LDS + j], S[i * LDS + k]);
      }
      __syncthreads();
    }
    // L_jj = sqrt(d_j), L_ij = S_ij / sqrt(d_j): one square root and one reciprocal per
    // column (warps 0 and 1), then products
    if (tid < T) {
      const double r = sqrt(s_d[tid]);
      s_d[tid] = r;
      s_rcp[tid] = 1.0 / r;
    }
    __syncthreads();
    for (int e = tid; e < T * T; e += kThreads) {
      const int i = e / T, j = e % T;
      if (j > i) continue;
      Di[i * LDS + j] = i == j ? s_d[j] : S[i * LDS + j] * s_rcp[j];  // L_KK, staged in Di
    }
    __syncthreads();
    for (int e = tid; e < T * T; e += kThreads) {
      const int i = e / T, j = e % T;
      S[i * LDS + j] = j <= i ? Di[i * LDS + j] : 0.0;
    }
    __syncthreads();
    // ---- 2. inv(L_KK) by rows: Di_ic = (delta_ic - sum_{c<=k<i} L_ik Di_kc) / L_ii; row i
    // depends on rows < i only, so all columns c of a row run in parallel (4 threads per
    // column split the sum, fixed-order shuffle reduction)
    {
      // 1 / L_ii of every row is s_rcp (computed above from the same sqrt(d_i))
      const int c = tid >> 2, q = tid & 3;
      for (int i = 0; i < T; ++i) {
        double acc = 0.0;
        if (c < i)
          for (int k = c + q; k < i; k += 4) acc = fma(S[i * LDS + k], Di[k * LDS + c], acc);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (q == 0) {
          const double ri = s_rcp[i];
          Di[i * LDS + c] = c < i ? -acc * ri : (c == i ? ri : 0.0);
        }
        __syncthreads();
      }
    }
    // write L_KK (upper part zeroed) and inv(L_KK)
    double *dK = dinv + B.dinv_off + (int64_t)K * T * T;
    for (int e = tid; e < T * T; e += kThreads) {
      const int r = e / T, c = e % T;
      gKK[e] = c <= r ? S[r * LDS + c] : 0.0;
      dK[e] = c <= r ? Di[r * LDS + c] : 0.0;
    }
    __syncthreads();  // L_KK and inv(L_KK) are in global memory; S / Di are free
    // Bt[k][c] = inv(L_KK)(c, k) for the TRSM below (upper triangle: unit column block C
    // needs k < 16 (C + 1)); read back from dinv (L1-resident)
    load_kmajor(dK, Bt);
    __syncthreads();
    // ---- 3. L_IK = G_IK * Di^T for every stored tile below the diagonal
    for (int I = K + 1; I < B.nt; ++I) {
      const TileRow TI = tr[I];
      if (TI.j0 > K) continue;
      double *gIK = tile_ptr(fac, TI, K);
      load_kmajor(gIK, At);
      __syncthreads();
      for (int u = warp; u < 16; u += kWarps) {
        const int R = u >> 2, C = u & 3;
        double acc[2][4];
        unit_product(At, Bt, R, C, 16 * (C + 1), acc);
        unit_store(gIK, R, C, acc, false);
      }
      __syncthreads();
    }
    // ---- 4. trailing update G_IJ -= L_IK L_JK^T; a diagonal tile (J = I) is symmetric and
    // only its lower units are updated (the upper triangle of G_II is never read)
    for (int I = K + 1; I < B.nt; ++I) {
      const TileRow TI = tr[I];
      if (TI.j0 > K) continue;
      load_kmajor(tile_ptr(fac, TI, K), At);
      for (int J = K + 1; J <= I; ++J) {
        const TileRow TJ = tr[J];
        if (TJ.j0 > K) continue;
        __syncthreads();  // previous use of Bt finished
        load_kmajor(tile_ptr(fac, TJ, K), Bt);
        __syncthreads();
        double *gIJ = tile_ptr(fac, TI, J);
        if (J < I) {
          for (int u = warp; u < 16; u += kWarps) {
            const int R = u >> 2, C = u & 3;
            double acc[2][4];
            unit_product(At, Bt, R, C, T, acc);
            unit_store(gIJ, R, C, acc, true);
          }
        } else {
          for (int u = warp; u < 10; u += kWarps) {
            int R, C;
            lower_unit(u, R, C);
            double acc[2][4];
            unit_product(At, Bt, R, C, T, acc);
            unit_store(gIJ, R, C, acc, true);
          }
        }
      }
      __syncthreads();
    }
    __syncthreads();
  }
  if (tid == 0) {
    pivmin[b] = s_pmin;
    pivfail[b] = s_fail;
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
// blocks (one CTA per block and tile row); inv(L_KK) is lower triangular, so unit row block R
// needs k < 16 (R + 1).
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
  const int warp = threadIdx.x >> 5;
  load_kmajor(dinv + B.dinv_off + (int64_t)K * T * T, At);
  for (int J = TK.j0; J < K; ++J) {
    double *g = tile_ptr(fac, TK, J);
    __syncthreads();
    load_rowmajor(g, Bt);
    __syncthreads();
    for (int u = warp; u < 16; u += kWarps) {
      const int R = u >> 2, C = u & 3;
      double acc[2][4];
      unit_product(At, Bt, R, C, 16 * (R + 1), acc);
      unit_store(g, R, C, acc, false);
    }
  }
}

constexpr int kCholSmem = (int)sizeof(double) * 2 * T * LD;
// dynamic shared memory requested by k_cholesky: more than half of an SM's 228 KB, so that
// one block runs per SM (measured fastest, see the header)
constexpr int kCholSmemLaunch = 120 * 1024;
static_assert(T * LDS <= T * LD, "diagonal scratch inside an operand tile");
static_assert(kCholSmemLaunch >= kCholSmem, "launch reservation covers the tiles");

}  // namespace

void launch_cholesky(const BlockDesc *blk, const int32_t *blist, int32_t nlist,
                     const TileRow *trow, double *fac, double *dinv, double *pivmin,
                     int32_t *pivfail, cudaStream_t s) {
  if (nlist <= 0) return;
  cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, kCholSmemLaunch);
  k_cholesky<<<(unsigned)nlist, kThreads, kCholSmemLaunch, s>>>(blk, blist, trow, fac, dinv,
                                                               pivmin, pivfail);
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
