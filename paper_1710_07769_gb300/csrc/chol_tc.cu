// Batched Cholesky of FP32 Gram blocks with the trailing update on the tensor cores.
//
// Same right-looking tile algorithm (and the same stored form L = diag(L_II)(I + N)) as
// the CUDA-core kernel in chol_kernels.cu; only step 4, the trailing update
//     G_IJ -= L_IK L_JK^T     for K < J <= I,
// the one dense contraction of the method, runs as tcgen05 MMAs:
//   * A = [L_{I0,K}; L_{I0+1,K}] (128 x 64, two tile rows), B = [L_{J0,K}; L_{J0+1,K}]
//     (128 x 64, two tile columns), D = A B^T (128 x 128, FP32) in tensor memory;
//   * 3xTF32 for FP32-level accuracy: x = hi + lo with hi = x rounded to TF32 and
//     lo = x - hi, D = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T (the TF32 operands are
//     read from shared memory in the canonical no-swizzle K-major layout: 8-row x
//     16-byte core matrices, 128 bytes apart along K, 2048 bytes apart along rows);
//   * one thread issues the 24 MMAs (K = 8 each) and commits them to an mbarrier; the
//     8 warps read D back with tcgen05.ld (warp w: lanes 32 (w mod 4).., half of the
//     columns) and subtract it from the tiles in global memory.
// Tiles outside the envelope read as zero and are never written.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace cimmino {

namespace {

constexpr int T = kTile;
constexpr int kThreads = 256;
constexpr int LDS = T + 1;  // padded row-major diagonal tile
constexpr int LD = T + 1;   // k-major operand tiles of the CUDA-core steps (odd: the
                            // transposed stores hit 32 distinct banks)
constexpr uint32_t kCoreK = 128;    // bytes between core matrices along K
constexpr uint32_t kCoreRow = 2048; // bytes between 8-row groups (16 core matrices of K = 64)
constexpr uint32_t kTmemCols = 128;
constexpr int kDstLd = 132;  // padded row of the epilogue staging area (floats)
constexpr uint64_t kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(kCoreK >> 4) << 16;    // leading (K) byte offset
  d |= (uint64_t)(kCoreRow >> 4) << 32;  // stride (row) byte offset
  d |= (uint64_t)1 << 46;                // descriptor version; no swizzle
  return d;
}
// D f32, A/B tf32, both K-major, M = 128, N = 128 (trailing update) or 64 (TRSM)
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) |
                            ((128u >> 4) << 24);
constexpr uint32_t kIdescN64 = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) |
                               ((128u >> 4) << 24);
constexpr int kStLd = T + 4;  // padded row of the TRSM epilogue staging area (floats)

// byte offset of element (r, k) of a 128 x 64 operand in the canonical layout
__device__ __forceinline__ uint32_t canon(int r, int k) {
  return (uint32_t)((r >> 3) * kCoreRow + (k >> 2) * kCoreK + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return __uint_as_float(h);
}

// Fill a 128 x 64 hi/lo operand pair from two row-major tiles (rows 0..63 from g0, rows
// 64..127 from g1; a null tile reads as zeros).  A warp handles 8 rows x 4 16-byte chunks
// per unit: lane l takes row 8 rg + (l & 7), chunk 4 cq + (l >> 3), so each quarter-warp
// stores one whole 128-byte core matrix (conflict-free) and reads 8 rows x 64 contiguous
// bytes from global memory.  All 8 loads of a lane are issued before the first store.
__device__ __forceinline__ void load_split2(const float *__restrict__ g0,
                                            const float *__restrict__ g1, unsigned char *hi,
                                            unsigned char *lo) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int U = 32 / (kThreads / 32);  // units per warp and tile
  float4 x[2][U];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float *g = h ? g1 : g0;
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int u = warp + (kThreads / 32) * j;
      const int r = 8 * (u >> 2) + (lane & 7), kc = 4 * (u & 3) + (lane >> 3);
      x[h][j] = g ? *reinterpret_cast<const float4 *>(g + r * T + 4 * kc)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int u = warp + (kThreads / 32) * j;
      const int r = 8 * (u >> 2) + (lane & 7), kc = 4 * (u & 3) + (lane >> 3);
      const float4 v = x[h][j];
      const float4 t = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
      const uint32_t o =
          (uint32_t)(((64 * h + r) >> 3) * kCoreRow + kc * kCoreK + (r & 7) * 16);
      *reinterpret_cast<float4 *>(hi + o) = t;
      *reinterpret_cast<float4 *>(lo + o) = make_float4(v.x - t.x, v.y - t.y, v.z - t.z, v.w - t.w);
    }
}

// Transposed operand layout (second canonical no-swizzle K-major form): core matrices of
// 8 rows x 16 bytes, 8-row groups 128 bytes apart, K chunks of 4 values 2048 bytes apart.
constexpr uint32_t kTCoreK = 2048;  // bytes between core matrices along K
constexpr uint32_t kTCoreRow = 128; // bytes between 8-row groups
__device__ __forceinline__ uint64_t smem_desc_t(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(kTCoreK >> 4) << 16;
  d |= (uint64_t)(kTCoreRow >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// B operand rows 0..63 = columns of g0, rows 64..127 = columns of g1 (B[n][k] = g[k][n]),
// hi/lo split, in the transposed layout: in every step a warp stores 8 rows x 4 k values,
// 32 consecutive words (conflict-free); the loads read 4 rows x 32 contiguous bytes.
__device__ __forceinline__ void load_split2_t(const float *__restrict__ g0,
                                              const float *__restrict__ g1, unsigned char *hi,
                                              unsigned char *lo) {
  const int tid = threadIdx.x, kk = tid & 3;
  constexpr int IT = 128 * T / kThreads;  // 32 values per thread
#pragma unroll 4
  for (int h = 0; h < IT; h += 8) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int it = h + j, k4 = it & 15, n = (tid >> 2) + 64 * (it >> 4);
      const float *g = n < 64 ? g0 : g1;
      x[j] = g ? g[(4 * k4 + kk) * T + (n & 63)] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int it = h + j, k4 = it & 15, n = (tid >> 2) + 64 * (it >> 4);
      const uint32_t o = (uint32_t)(k4 * kTCoreK + (n >> 3) * kTCoreRow + (n & 7) * 16 + kk * 4);
      const float t = tf32_hi(x[j]);
      *reinterpret_cast<float *>(hi + o) = t;
      *reinterpret_cast<float *>(lo + o) = x[j] - t;
    }
  }
}

__device__ __forceinline__ float *tile_ptr(float *fac, const TileRow &tr, int J) {
  return fac + tr.off + (int64_t)(J - tr.j0) * T * T;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc,
                                         uint32_t idesc = kIdesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

// One thread issues D = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T over K = 64 (3xTF32, 24
// MMAs) and commits them to mbar; every thread then waits for the commit (bounded: about
// 2 s, after which s_err and bit 4 of the error word are set and the kernel winds down).
// BT: B is in the transposed layout (smem_desc_t, K chunks kTCoreK apart).
template <bool BT = false>
__device__ __forceinline__ void mma_3xtf32(uint32_t tmem, const unsigned char *Ahi,
                                           const unsigned char *Alo, const unsigned char *Bhi,
                                           const unsigned char *Blo, uint32_t idesc,
                                           uint64_t *mbar, uint32_t &phase, int *s_err,
                                           int32_t *err) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x == 0) {
    const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
    for (int s = 0; s < T / 8; ++s) {
      const uint32_t ko = s * 2 * kCoreK;  // K = 8 per MMA: two core matrices
      const uint32_t kb = s * 2 * (BT ? kTCoreK : kCoreK);
      const uint64_t bdh = BT ? smem_desc_t(bh + kb) : smem_desc(bh + kb);
      const uint64_t bdl = BT ? smem_desc_t(bl + kb) : smem_desc(bl + kb);
      mma_tf32(tmem, smem_desc(ah + ko), bdh, s > 0, idesc);
      mma_tf32(tmem, smem_desc(ah + ko), bdl, 1, idesc);
      mma_tf32(tmem, smem_desc(al + ko), bdh, 1, idesc);
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(mbar))
        : "memory");
  }
  uint32_t ok = 0;
  const uint64_t t0 = global_ns();
  while (!ok) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(phase)
        : "memory");
    if (!ok && global_ns() - t0 > kWaitNs) {
      *s_err = 1;
      atomicOr(err, 4);
      break;
    }
  }
  phase ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,"
      "%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,"
      "%61,%62,%63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]),
        "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]),
        "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
        "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]),
        "=r"(r[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 64; ++j) v[j] = __uint_as_float(r[j]);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_cholesky_tc(const BlockDesc *__restrict__ blk, const int32_t *__restrict__ blist,
                  const TileRow *__restrict__ trow, float *__restrict__ fac,
                  float *__restrict__ dinv, double *__restrict__ pivmin,
                  int32_t *__restrict__ pivfail, int32_t *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *Ahi = smem_raw;          // 128 x 64 TF32 operands, 32 KB each
  unsigned char *Alo = Ahi + 32768;
  unsigned char *Bhi = Alo + 32768;
  unsigned char *Blo = Bhi + 32768;
  float *At = reinterpret_cast<float *>(Blo + 32768);  // [T][LD]
  float *Bt = At + T * LD;                             // [T][LD]
  float *S = Bt + T * LD;                              // [T][LDS]
  float *Di = S + T * LDS;                             // [T][LDS]
  float *Dst = reinterpret_cast<float *>(Bhi);  // [128][kDstLd] epilogue staging (B, At)
  float *St = At;  // [128][kStLd] TRSM epilogue staging (At, Bt, S)
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ double s_pmin;
  __shared__ int s_fail, s_err;

  const int b = blist[blockIdx.x];
  const BlockDesc B = blk[b];
  const TileRow *tr = trow + B.trow0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tr4 = tid / 16, tc4 = tid % 16;
  if (tid == 0) {
    s_pmin = 1e300;
    s_fail = 0;
    s_err = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  uint32_t phase = 0;

  for (int K = 0; K < B.nt && !s_err; ++K) {
    const TileRow TK = tr[K];
    float *gKK = tile_ptr(fac, TK, K);
    // ---- 1. diagonal tile (CUDA cores), right-looking with the column scaling deferred:
    // step j subtracts S_ij S_kj / d_j from the trailing triangle (one barrier per column);
    // afterwards L_jj = sqrt(d_j) and L_ij = S_ij / sqrt(d_j)
    for (int e = tid; e < T * T; e += kThreads) S[(e / T) * LDS + (e % T)] = gKK[e];
    __syncthreads();
    for (int j = 0; j < T; ++j) {
      float dj = S[j * LDS + j];
      if (tid == 0 && K * T + j < B.m) s_pmin = fmin(s_pmin, (double)dj);
      if (!(dj > 0.f) || !isfinite(dj)) {
        if (tid == 0) s_fail = 1;
        dj = 1.f;
      }
      const float inv = 1.f / dj;
      for (int i = j + 1 + tr4; i < T; i += 16) {
        const float t = S[i * LDS + j] * inv;
        for (int k = j + 1 + tc4; k <= i; k += 16) S[i * LDS + k] = fmaf(-t, S[k * LDS + j], S[i * LDS + k]);
      }
      __syncthreads();
    }
    for (int e = tid; e < T * T; e += kThreads) {
      const int i = e / T, j = e % T;
      if (j > i) continue;
      float dj = S[j * LDS + j];
      if (!(dj > 0.f) || !isfinite(dj)) dj = 1.f;
      Di[i * LDS + j] = i == j ? sqrtf(dj) : S[i * LDS + j] / sqrtf(dj);  // L_KK, staged in Di
    }
    __syncthreads();
    for (int e = tid; e < T * T; e += kThreads) {
      const int i = e / T, j = e % T;
      S[i * LDS + j] = j <= i ? Di[i * LDS + j] : 0.f;
    }
    __syncthreads();
    // ---- 2. inv(L_KK) by rows: Di_ic = (delta_ic - sum_{c<=k<i} L_ik Di_kc) / L_ii; row i
    // depends on rows < i only, so all columns c of a row run in parallel (4 threads per
    // column split the sum, fixed-order shuffle reduction)
    {
      const int c = tid >> 2, q = tid & 3;
      for (int i = 0; i < T; ++i) {
        float acc = 0.f;
        if (c < i)
          for (int k = c + q; k < i; k += 4) acc = fmaf(S[i * LDS + k], Di[k * LDS + c], acc);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (q == 0) {
          const float lii = S[i * LDS + i];
          Di[i * LDS + c] = c < i ? -acc / lii : (c == i ? 1.f / lii : 0.f);
        }
        __syncthreads();
      }
    }
    float *dK = dinv + B.dinv_off + (int64_t)K * T * T;
    for (int e = tid; e < T * T; e += kThreads) {
      int r = e / T, c = e % T;
      gKK[e] = c <= r ? S[r * LDS + c] : 0.f;
      dK[e] = c <= r ? Di[r * LDS + c] : 0.f;
    }
    // N_KJ = inv(L_KK) L_KJ for the final row K on the tensor cores, pairs of tiles:
    // D (128 x 128) = [inv(L_KK); 0] [L_KJ0 L_KJ1] (rows 64..127 of A are zero, so half of
    // D is unused), A = inv(L_KK) read back from dK, B row n = column n of the pair in the
    // transposed layout; rows 0..63 of D go through the padded staging area (At, Bt, S)
    __syncthreads();  // dK is complete
    if (TK.j0 < K) load_split2(dK, nullptr, Ahi, Alo);
    for (int J0 = TK.j0; J0 < K && !s_err; J0 += 2) {
      const bool has1 = J0 + 1 < K;
      float *g0 = tile_ptr(fac, TK, J0);
      float *g1 = has1 ? tile_ptr(fac, TK, J0 + 1) : nullptr;
      load_split2_t(g0, g1, Bhi, Blo);
      mma_3xtf32<true>(tmem, Ahi, Alo, Bhi, Blo, kIdesc, &mbar, phase, &s_err, err);
      if ((warp & 3) < 2) {  // TMEM lanes 0..63 (warps 0, 1, 4, 5), column half warp / 4
        const int rr = 32 * (warp & 3) + lane, jh = warp >> 2;
        float v[64];
        tmem_ld64(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * jh), v);
        float *st = St + rr * kDstLd + 64 * jh;
#pragma unroll
        for (int c = 0; c < 64; c += 4)
          *reinterpret_cast<float4 *>(st + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
      }
      __syncthreads();
      if (!s_err) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          float *gq = q ? g1 : g0;
          if (!gq) continue;
          for (int e = tid; e < T * T / 4; e += kThreads) {
            const int r = e >> 4, c = 4 * (e & 15);
            *reinterpret_cast<float4 *>(gq + r * T + c) =
                *reinterpret_cast<const float4 *>(St + r * kDstLd + 64 * q + c);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    // ---- 3. L_IK = G_IK inv(L_KK)^T on the tensor cores, pairs of tile rows:
    // D (128 x 64) = [G_I0K; G_I1K] inv(L_KK)^T, i.e. B = inv(L_KK) (K-major rows, read
    // back from dK); D goes through a padded staging area (the CUDA-core scratch At, Bt,
    // S, free by now) into coalesced 16-byte stores
    __syncthreads();  // dK is complete
    load_split2(dK, nullptr, Bhi, Blo);
    for (int I0 = K + 1; I0 < B.nt && !s_err; I0 += 2) {
      const int I1 = I0 + 1;
      const bool has0 = tr[I0].j0 <= K;
      const bool has1 = I1 < B.nt && tr[I1].j0 <= K;
      if (!has0 && !has1) continue;
      float *g0 = has0 ? tile_ptr(fac, tr[I0], K) : nullptr;
      float *g1 = has1 ? tile_ptr(fac, tr[I1], K) : nullptr;
      load_split2(g0, g1, Ahi, Alo);
      mma_3xtf32(tmem, Ahi, Alo, Bhi, Blo, kIdescN64, &mbar, phase, &s_err, err);
      if (warp < 4) {  // warp w reads TMEM lanes 32 w .. 32 w + 31, columns 0..63
        const int rr = 32 * warp + lane;
        float v[64];
        tmem_ld64(tmem + ((uint32_t)(32 * warp) << 16), v);
        float *st = St + rr * kStLd;
#pragma unroll
        for (int c = 0; c < 64; c += 4)
          *reinterpret_cast<float4 *>(st + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
      }
      __syncthreads();
      if (!s_err) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          float *gq = q ? g1 : g0;
          if (!gq) continue;
          for (int e = tid; e < T * T / 4; e += kThreads) {
            const int r = e >> 4, c = 4 * (e & 15);
            *reinterpret_cast<float4 *>(gq + r * T + c) =
                *reinterpret_cast<const float4 *>(St + (64 * q + r) * kStLd + c);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    // ---- 4. trailing update on the tensor cores: pairs of tile rows x pairs of tile columns
    for (int I0 = K + 1; I0 < B.nt && !s_err; I0 += 2) {
      const int I1 = I0 + 1;
      const bool has0 = tr[I0].j0 <= K;
      const bool has1 = I1 < B.nt && tr[I1].j0 <= K;
      if (!has0 && !has1) continue;
      load_split2(has0 ? tile_ptr(fac, tr[I0], K) : nullptr,
                  has1 ? tile_ptr(fac, tr[I1], K) : nullptr, Ahi, Alo);
      const int jmax = has1 ? I1 : I0;
      for (int J0 = K + 1; J0 <= jmax && !s_err; J0 += 2) {
        const int J1 = J0 + 1;
        const bool hj0 = tr[J0].j0 <= K;
        const bool hj1 = J1 <= jmax && J1 < B.nt && tr[J1].j0 <= K;
        if (!hj0 && !hj1) continue;
        load_split2(hj0 ? tile_ptr(fac, tr[J0], K) : nullptr,
                    hj1 ? tile_ptr(fac, tr[J1], K) : nullptr, Bhi, Blo);
        mma_3xtf32(tmem, Ahi, Alo, Bhi, Blo, kIdesc, &mbar, phase, &s_err, err);
        // epilogue: warp w reads lanes 32 (w mod 4).. and column half w / 4 of D into the
        // staging area (the B operands, free once the MMAs completed; rows padded to 132
        // floats so that a quarter-warp's 16-byte stores hit 8 distinct bank groups), then
        // all threads update the four global tiles with coalesced 16-byte read-modify-writes
        {
          const int rowq = warp & 3, jh = warp >> 2;
          const int rr = 32 * rowq + lane;  // row of D
          float v[64];
          tmem_ld64(tmem + ((uint32_t)(32 * rowq) << 16) + (uint32_t)(64 * jh), v);
          float *st = Dst + rr * kDstLd + 64 * jh;
#pragma unroll
          for (int c = 0; c < 64; c += 4)
            *reinterpret_cast<float4 *>(st + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
        }
        __syncthreads();
        if (!s_err) {
          // tile (I, J) of quadrant q: q & 1 -> I1, q >> 1 -> J1; all 16 loads of a thread
          // are in flight before the first subtraction
          constexpr int R = T * T / 4 / kThreads;  // 16-byte chunks per thread and tile
          float *gq[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int I = (q & 1) ? I1 : I0, J = (q >> 1) ? J1 : J0;
            const bool ok = ((q & 1) ? has1 : has0) && ((q >> 1) ? hj1 : hj0) && J <= I;
            gq[q] = ok ? tile_ptr(fac, tr[I], J) : nullptr;
          }
          float4 x[4][R];
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int j = 0; j < R; ++j) {
              const int e = tid + kThreads * j, r = e >> 4, c = 4 * (e & 15);
              if (gq[q]) x[q][j] = *reinterpret_cast<const float4 *>(gq[q] + r * T + c);
            }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (!gq[q]) continue;
            const float *src = Dst + 64 * (q & 1) * kDstLd + 64 * (q >> 1);
#pragma unroll
            for (int j = 0; j < R; ++j) {
              const int e = tid + kThreads * j, r = e >> 4, c = 4 * (e & 15);
              const float4 d = *reinterpret_cast<const float4 *>(src + r * kDstLd + c);
              float4 v = x[q][j];
              v.x -= d.x;
              v.y -= d.y;
              v.z -= d.z;
              v.w -= d.w;
              *reinterpret_cast<float4 *>(gq[q] + r * T + c) = v;
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    pivmin[b] = s_pmin;
    pivfail[b] = s_fail | s_err;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

constexpr int kTcSmem = 4 * 32768 + (int)sizeof(float) * (2 * T * LD + 2 * T * LDS);
// the epilogue staging area (128 x kDstLd floats from Bhi) fits in Bhi, Blo and At; the
// TRSM staging area (128 x kStLd floats from At) in At, Bt and S, short of Di
static_assert(128 * kDstLd * 4 <= 2 * 32768 + (int)sizeof(float) * T * LD, "staging area");
static_assert(128 * kStLd <= 2 * T * LD + T * LDS, "TRSM staging area");
static_assert(64 * kDstLd <= 2 * T * LD + T * LDS, "N-transform staging area");

}  // namespace

void launch_cholesky_tc(const BlockDesc *blk, const int32_t *blist, int32_t nlist,
                        const TileRow *trow, float *fac, float *dinv, double *pivmin,
                        int32_t *pivfail, int32_t *err, cudaStream_t s) {
  if (nlist <= 0) return;
  cudaFuncSetAttribute(k_cholesky_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  k_cholesky_tc<<<(unsigned)nlist, kThreads, kTcSmem, s>>>(blk, blist, trow, fac, dinv, pivmin,
                                                           pivfail, err);
}

}  // namespace cimmino
