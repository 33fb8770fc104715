// Batched Cholesky G_i = L_i L_i^T of the Gram blocks, in place on the tiled
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
// pivot is replaced by 1 so that the block finishes without NaNs and can be
// refactored in FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace cimmino {

namespace {

constexpr int T = kTile;
constexpr int kThreads = 256;

template <typename W>
struct Pad {
  static constexpr int v = 16 / sizeof(W);  // keeps k-major rows 16-byte aligned
};

template <typename W>
__device__ __forceinline__ W *tile_ptr(W *fac, const TileRow &tr, int J) {
  return fac + tr.off + (int64_t)(J - tr.j0) * T * T;
}

// Load a row-major global tile into k-major shared storage At[k][r] = tile(r, k).
template <typename W>
__device__ __forceinline__ void load_kmajor(const W *__restrict__ g, W *At) {
  constexpr int LD = T + Pad<W>::v;
  for (int e = threadIdx.x; e < T * T; e += kThreads) {
    int r = e / T, k = e % T;
    At[k * LD + r] = g[e];
  }
}

// acc(r, c) for the thread's 4 x 4 block: sum_k At[k][r] * Bt[k][c]
template <typename W>
__device__ __forceinline__ void mma_4x4(const W *At, const W *Bt, W acc[4][4]) {
  constexpr int LD = T + Pad<W>::v;
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
#pragma unroll 8
  for (int k = 0; k < T; ++k) {
    W a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = At[k * LD + tr * 4 + i];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Bt[k * LD + tc * 4 + j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
}

template <typename W>
__global__ void __launch_bounds__(kThreads)
    k_cholesky(const BlockDesc *__restrict__ blk, const int32_t *__restrict__ blist,
               const TileRow *__restrict__ trow, W *__restrict__ fac, W *__restrict__ dinv,
               double *__restrict__ pivmin, int32_t *__restrict__ pivfail) {
  constexpr int LDS = T + 1;            // padded row-major diagonal tile
  constexpr int LD = T + Pad<W>::v;     // k-major operand tiles
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W *At = reinterpret_cast<W *>(smem_raw);  // [T][LD]
  W *Bt = At + T * LD;                      // [T][LD]
  W *S = Bt + T * LD;                       // [T][LDS]
  W *Di = S + T * LDS;                      // [T][LDS]
  __shared__ double s_pmin;
  __shared__ int s_fail;

  const int b = blist[blockIdx.x];
  const BlockDesc B = blk[b];
  const TileRow *tr = trow + B.trow0;
  const int tid = threadIdx.x;
  const int tr4 = tid / 16, tc4 = tid % 16;
  if (tid == 0) {
    s_pmin = 1e300;
    s_fail = 0;
  }
  __syncthreads();

  for (int K = 0; K < B.nt; ++K) {
    const TileRow TK = tr[K];
    W *gKK = tile_ptr(fac, TK, K);
    // ---- 1. diagonal tile: unblocked right-looking Cholesky in shared memory
    for (int e = tid; e < T * T; e += kThreads) S[(e / T) * LDS + (e % T)] = gKK[e];
    __syncthreads();
    for (int j = 0; j < T; ++j) {
      if (tid == 0) {
        W dj = S[j * LDS + j];
        if (K * T + j < B.m) s_pmin = fmin(s_pmin, (double)dj);
        if (!(dj > W(0)) || !isfinite((double)dj)) {
          s_fail = 1;
          dj = W(1);
        }
        S[j * LDS + j] = sqrt(dj);
      }
      __syncthreads();
      const W ljj = S[j * LDS + j];
      for (int i = j + 1 + tid; i < T; i += kThreads) S[i * LDS + j] = S[i * LDS + j] / ljj;
      __syncthreads();
      const int w = T - j - 1;
      for (int e = tid; e < w * w; e += kThreads) {
        int i = j + 1 + e / w, k = j + 1 + e % w;
        if (k <= i) S[i * LDS + k] = fma(-S[i * LDS + j], S[k * LDS + j], S[i * LDS + k]);
      }
      __syncthreads();
    }
    // ---- 2. Di = inv(L_KK), column by column (forward substitution on unit vectors)
    if (tid < T) {
      const int c = tid;
      for (int i = 0; i < c; ++i) Di[i * LDS + c] = W(0);
      Di[c * LDS + c] = W(1) / S[c * LDS + c];
      for (int i = c + 1; i < T; ++i) {
        W s = W(0);
        for (int k = c; k < i; ++k) s = fma(S[i * LDS + k], Di[k * LDS + c], s);
        Di[i * LDS + c] = -s / S[i * LDS + i];
      }
    }
    __syncthreads();
    // write L_KK (upper part zeroed) and inv(L_KK)
    W *dK = dinv + B.dinv_off + (int64_t)K * T * T;
    for (int e = tid; e < T * T; e += kThreads) {
      int r = e / T, c = e % T;
      gKK[e] = c <= r ? S[r * LDS + c] : W(0);
      dK[e] = c <= r ? Di[r * LDS + c] : W(0);
    }
    // Row K is final now: store N_KJ = inv(L_KK) L_KJ in place of L_KJ (J < K), so that
    // the solves see L = diag(L_II) (I + N) and their sequential chains need no
    // diagonal solve.  At[k][r] = Di(r, k), Bt[k][c] = L_KJ(k, c).
    for (int e = tid; e < T * T; e += kThreads) {
      int k = e / T, r = e % T;
      At[k * LD + r] = Di[r * LDS + k];
    }
    for (int J = TK.j0; J < K; ++J) {
      W *gKJ = tile_ptr(fac, TK, J);
      __syncthreads();  // At ready / previous use of Bt finished
      for (int e = tid; e < T * T; e += kThreads) Bt[(e / T) * LD + (e % T)] = gKJ[e];
      __syncthreads();
      W acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = W(0);
      mma_4x4(At, Bt, acc);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) gKJ[(tr4 * 4 + i) * T + tc4 * 4 + j] = acc[i][j];
    }
    __syncthreads();
    // Bt[k][c] = Di(c, k) for the TRSM below
    for (int e = tid; e < T * T; e += kThreads) {
      int k = e / T, c = e % T;
      Bt[k * LD + c] = Di[c * LDS + k];
    }
    __syncthreads();
    // ---- 3. L_IK = G_IK * Di^T for every stored tile below the diagonal
    for (int I = K + 1; I < B.nt; ++I) {
      const TileRow TI = tr[I];
      if (TI.j0 > K) continue;
      W *gIK = tile_ptr(fac, TI, K);
      load_kmajor(gIK, At);
      __syncthreads();
      W acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = W(0);
      mma_4x4(At, Bt, acc);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) gIK[(tr4 * 4 + i) * T + tc4 * 4 + j] = acc[i][j];
      __syncthreads();
    }
    // ---- 4. trailing update G_IJ -= L_IK L_JK^T
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
        W *gIJ = tile_ptr(fac, TI, J);
        W acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = W(0);
        mma_4x4(At, Bt, acc);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            W *p = gIJ + (tr4 * 4 + i) * T + tc4 * 4 + j;
            *p = *p - acc[i][j];
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
  for (int I = 0; I < B.nt; ++I) {
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

template <typename W>
int chol_smem() {
  return (int)(sizeof(W) * (2 * T * (T + Pad<W>::v) + 2 * T * (T + 1)));
}

}  // namespace

void launch_cholesky(const BlockDesc *blk, const int32_t *blist, int32_t nlist,
                     const TileRow *trow, void *fac, void *dinv, int prec64, double *pivmin,
                     int32_t *pivfail, cudaStream_t s) {
  if (nlist <= 0) return;
  if (prec64) {
    int sm = chol_smem<double>();
    cudaFuncSetAttribute(k_cholesky<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    k_cholesky<double><<<(unsigned)nlist, kThreads, sm, s>>>(
        blk, blist, trow, static_cast<double *>(fac), static_cast<double *>(dinv), pivmin,
        pivfail);
  } else {
    int sm = chol_smem<float>();
    cudaFuncSetAttribute(k_cholesky<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    k_cholesky<float><<<(unsigned)nlist, kThreads, sm, s>>>(
        blk, blist, trow, static_cast<float *>(fac), static_cast<float *>(dinv), pivmin,
        pivfail);
  }
}

void launch_transpose_factor(const BlockDesc *blk, int32_t nblk, const TileRow *trow,
                             const TileRow *trowT, const FactorPtrs &f, cudaStream_t s) {
  if (nblk > 0) k_transpose_factor<<<(unsigned)nblk, kThreads, 0, s>>>(blk, trow, trowT, f);
  if (nblk > 0) k_pack_diag<<<(unsigned)nblk, kThreads, 0, s>>>(blk, f);
}

}  // namespace cimmino
