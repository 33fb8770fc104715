// Batched Cholesky of FP32 Gram blocks on the tensor cores, left-looking.
//
// One CTA per block; for every tile column K (the panel) of L_i:
//   1. accumulate  D_I = sum_{J < K} L_IJ L_KJ^T  for every panel row I >= K inside the
//      envelope, in tensor memory: rows are taken in pairs (M = 128: tiles I0, I1), the
//      panel is one tile wide (N = 64), K-dimension 64 per tile J;
//   2. factor the diagonal tile: L_KK L_KK^T = G_KK - D_K (CUDA cores), and invert L_KK;
//   3. L_IK = (G_IK - D_I) inv(L_KK)^T for the other panel rows (tensor cores again).
// The trailing matrix is never written back: every L tile is written once (to the factor
// and, split for the tensor cores, to a scratch copy), every G tile read once.  Row K of L
// is turned into N_KJ = inv(L_KK) L_KJ afterwards by a separate kernel (all tiles are
// independent there), which gives the stored form L = diag(L_II)(I + N).
//
// FP32 accuracy from TF32 tensor cores by the 3xTF32 split: x = hi + lo, hi = x rounded to
// TF32, lo = x - hi, and A B^T = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T.  The scratch copy
// holds every finished L tile as its hi and lo parts in the canonical no-swizzle K-major
// layout of the MMA operands (8-row x 16-byte core matrices, 128 bytes apart along K, 1024
// bytes apart along rows), cut into two K-halves of 32 columns: one bulk copy per 8 KB
// piece fills an operand stage.
//
// Roles (192 threads): warps 0-3 read and write tensor memory (thread t = accumulator row t)
// and do the CUDA-core work; warp 4 issues the bulk copies of the operand ring (two A stages
// of 32 KB: a row pair's K-half, hi and lo; two B stages of 16 KB: tile L_KJ's K-half); warp
// 5 issues the MMAs.  About 96 KB of shared memory and 256 tensor-memory columns (four
// 128 x 64 accumulators) per CTA, so two CTAs (two blocks) share an SM.  Every wait is
// bounded by %globaltimer: after about 2 s a role sets the abort flag and bit 4 of the error
// word, and every later wait returns at once, so the kernel always ends.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace cimmino {

namespace {

constexpr int T = kTile;
constexpr int kEpi = 128;                 // epilogue / CUDA-core threads (warps 0-3)
constexpr int kThreads = kEpi + 64;       // + producer warp + MMA warp
constexpr int kPairsMax = 4;              // accumulators per pass
constexpr uint32_t kTmemCols = 64 * kPairsMax;
constexpr uint32_t kHalf = 8192;          // bytes of one K-half image (64 rows x 32 x 4 B)
constexpr uint32_t kAStage = 4 * kHalf;   // [I0 hi][I1 hi][I0 lo][I1 lo]
constexpr uint32_t kBStage = 2 * kHalf;   // [hi][lo]
constexpr uint32_t kRing = 2 * kAStage + 2 * kBStage;  // 96 KB
constexpr int LDS = T + 1;
constexpr uint64_t kWaitNs = 2000000000ull;
// D f32, A/B tf32, K-major, M = 128, N = 64
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) |
                            ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// no-swizzle K-major operand descriptor: core matrices 128 B apart along K (leading byte
// offset), 8-row groups `sbo` bytes apart (stride byte offset)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)(sbo >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return __uint_as_float(h);
}
// byte offset of (row r, column k) in an image of 32-column K-halves (row groups 1024 B
// apart); `half_bytes` separates the two K-halves
__device__ __forceinline__ uint32_t half_off(int r, int k) {
  return (uint32_t)((k >> 5) * kHalf + (r >> 3) * 1024 + ((k & 31) >> 2) * 128 + (r & 7) * 16 +
                    (k & 3) * 4);
}
// byte offset of (row r, column k) in a full-K image (row groups 2048 B apart)
__device__ __forceinline__ uint32_t full_off(int r, int k) {
  return (uint32_t)((r >> 3) * 2048 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

struct Ctl {
  uint64_t full_a[2], empty_a[2], full_b[2], empty_b[2];
  uint64_t acc_ready, trsm_ready, trsm_done;
  uint32_t tmem_base;
  int abort;
  int fail;
  double pmin;
};

// Bounded wait on a barrier phase; gives up (and makes every later wait give up) after
// about 2 s or once another role has given up.
__device__ __forceinline__ bool wait_phase(Ctl *c, uint64_t *b, uint32_t parity, int32_t *err) {
  if (*(volatile int *)&c->abort) return false;
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < (1u << 30); ++i) {
    if (mbar_try_wait(b, parity)) return true;
    if (*(volatile int *)&c->abort) return false;
    if (global_ns() - t0 > kWaitNs) break;
  }
  *(volatile int *)&c->abort = 1;
  atomicOr(err, 4);
  return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 3xTF32 product over `ksteps` steps of K = 8: D (+)= A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T.
// A: 128 rows, B: 64 rows; hi/lo parts at the given shared addresses; sbo = row-group stride.
__device__ __forceinline__ void mma_3x(uint32_t tmem, uint32_t ah, uint32_t al, uint32_t bh,
                                       uint32_t bl, uint32_t sbo, int ksteps, bool accumulate) {
  for (int s = 0; s < ksteps; ++s) {
    const uint32_t ko = s * 256;  // K = 8: two core matrices
    mma_tf32(tmem, smem_desc(ah + ko, sbo), smem_desc(bh + ko, sbo), accumulate || s > 0);
    mma_tf32(tmem, smem_desc(ah + ko, sbo), smem_desc(bl + ko, sbo), 1);
    mma_tf32(tmem, smem_desc(al + ko, sbo), smem_desc(bh + ko, sbo), 1);
  }
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

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Cholesky L L^T of the 64 x 64 SPD tile in S (lower part read; L written in place, upper part
// zeroed) and inv(L) into Di, by the 128 epilogue threads (t = 0..127), blocked in 16 x 16
// sub-blocks so that the 64 pivots need 12 CTA-wide barriers instead of one each:
//   for each block column k: one warp factors the diagonal sub-block (rows in registers,
//   columns of L passed by shuffles), the rows below solve against it (one thread per row),
//   the trailing lower triangle is updated;
// then the inverse: each warp inverts one diagonal sub-block (a lane per column, in
// registers), and the
// off-diagonal sub-blocks follow by distance d = i - k: Di_ik = -Di_ii sum_{k<=m<i} L_im Di_mk.
// pmin receives the smallest pivot of the first `rows` rows; a pivot that is not positive
// and finite sets *fail and is replaced by 1.  Tmp: 3 x 256 floats of scratch.
__device__ __noinline__ void diag_factor_blocked(float *S, float *Di, float *Tmp, int t, int rows,
                                    double *pmin, int *fail) {
  const int warp = t >> 5, lane = t & 31;
  float *rcp = Tmp;  // 1 / L_jj of the 64 pivots (Tmp is free until the off-diagonal inverse)
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int b0 = 16 * k;
    if (warp == 0) {
      // the 16 x 16 diagonal sub-block in registers: lane r (and its mirror r + 16) holds
      // row r; column jj of L reaches the other rows by shuffles instead of shared memory
      const int r = lane & 15;
      float a[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) a[c] = S[(b0 + r) * LDS + b0 + c];
      // smallest pivot and failure of this sub-block, in registers (one shared update after)
      float pm = INFINITY;
      bool bad = false;
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int j = b0 + jj;
        float d = __shfl_sync(0xffffffffu, a[jj], jj);
        if (j < rows) pm = fminf(pm, d);
        if (!(d > 0.f) || !isfinite(d)) {
          bad = true;
          d = 1.f;
        }
        const float rc = rsqrtf(d), l = d * rc;
        if (lane == jj) rcp[j] = rc;
        // selects, not branches: the lanes stay converged through the step
        a[jj] = r == jj ? l : (r > jj ? a[jj] * rc : a[jj]);
        // rank-1 update of the block's remaining lower triangle
        float lc[16];
#pragma unroll
        for (int c = jj + 1; c < 16; ++c) lc[c] = __shfl_sync(0xffffffffu, a[jj], c);
#pragma unroll
        for (int c = jj + 1; c < 16; ++c) a[c] = r >= c ? fmaf(-a[jj], lc[c], a[c]) : a[c];
      }
      if (lane < 16) {
#pragma unroll
        for (int c = 0; c < 16; ++c) S[(b0 + r) * LDS + b0 + c] = a[c];
      }
      if (lane == 0) {
        if (pm < INFINITY) *pmin = fmin(*pmin, (double)pm);
        if (bad) *fail = 1;
      }
    }
    epi_sync();
    // rows below: L_ik = S_ik L_kk^-T, forward substitution along the row, one thread per row
    const int i = b0 + 16 + t;
    if (i < T) {
      float x[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        float v = S[i * LDS + b0 + c];
#pragma unroll
        for (int m = 0; m < c; ++m) v = fmaf(-x[m], S[(b0 + c) * LDS + b0 + m], v);
        x[c] = v * rcp[b0 + c];
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) S[i * LDS + b0 + c] = x[c];
    }
    epi_sync();
    // trailing lower triangle: S_ic -= sum_m L_im L_cm over the block column
    const int n = T - b0 - 16;
    for (int e = t; e < n * n; e += kEpi) {
      const int ii = b0 + 16 + e / n, c = b0 + 16 + e % n;
      if (c > ii) continue;
      float v = S[ii * LDS + c];
#pragma unroll
      for (int m = 0; m < 16; ++m) v = fmaf(-S[ii * LDS + b0 + m], S[c * LDS + b0 + m], v);
      S[ii * LDS + c] = v;
    }
    epi_sync();
  }
  // zero the upper triangle of L
  for (int e = t; e < T * T; e += kEpi) {
    const int i = e / T, j = e % T;
    if (j > i) S[i * LDS + j] = 0.f;
  }
  // inverse of every diagonal sub-block: warp k, lane c < 16 owns column c, kept in registers
  // (entries above the diagonal are zero, so the sums may start at m = 0)
  {
    const int b0 = 16 * warp;
    const int c = lane & 15;
    float col[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float ri = rcp[b0 + i];
      float v = 0.f;
#pragma unroll
      for (int m = 0; m < i; ++m) v = fmaf(-S[(b0 + i) * LDS + b0 + m], col[m], v);
      col[i] = i < c ? 0.f : (i == c ? ri : v * ri);
    }
    if (lane < 16) {
#pragma unroll
      for (int i = 0; i < 16; ++i) Di[(b0 + i) * LDS + b0 + c] = col[i];
    }
  }
  // the upper triangle of Di
  for (int e = t; e < T * T; e += kEpi) {
    const int i = e / T, j = e % T;
    if (j > i) Di[i * LDS + j] = 0.f;
  }
  epi_sync();
  for (int d = 1; d < 4; ++d) {
    const int np = 4 - d;  // pairs (i, k = i - d), i = d..3
    // Tmp_p = sum_{k <= m < i} L_im Di_mk
    for (int e = t; e < np * 256; e += kEpi) {
      const int p = e >> 8, r = (e >> 4) & 15, c = e & 15;
      const int bi = d + p, bk = p;
      float v = 0.f;
      for (int m = 16 * bk; m < 16 * bi; ++m)
        v = fmaf(S[(16 * bi + r) * LDS + m], Di[m * LDS + 16 * bk + c], v);
      Tmp[e] = v;
    }
    epi_sync();
    // Di_ik = -Di_ii Tmp
    for (int e = t; e < np * 256; e += kEpi) {
      const int p = e >> 8, r = (e >> 4) & 15, c = e & 15;
      const int bi = d + p, bk = p;
      float v = 0.f;
#pragma unroll
      for (int m = 0; m < 16; ++m) v = fmaf(Di[(16 * bi + r) * LDS + 16 * bi + m], Tmp[(p << 8) + m * 16 + c], v);
      Di[(16 * bi + r) * LDS + 16 * bk + c] = -v;
    }
    epi_sync();
  }
}

// The panel of column K: rows I >= K whose envelope reaches column K, in pairs.
struct Panel {
  int rows[2 * 64];
  int n;
};

__device__ __forceinline__ int64_t tile_index(const TileRow &tr, int J) {
  return tr.off + (int64_t)(J - tr.j0) * T * T;  // element offset of tile (I, J)
}

__global__ void __launch_bounds__(kThreads, 2)
    k_cholesky_tc(const BlockDesc *__restrict__ blk, const int32_t *__restrict__ blist,
                  const TileRow *__restrict__ trow, float *__restrict__ fac,
                  float *__restrict__ dinv, float *__restrict__ lc,
                  const float *__restrict__ zero_img, double *__restrict__ pivmin,
                  int32_t *__restrict__ pivfail, int32_t *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ Ctl ctl;
  __shared__ int s_rows[T];  // panel rows (a block has at most 64 tile rows)
  __shared__ int s_nrows;
  __shared__ TileRow s_tr[T];  // the block's tile-row table, read on every dependent step
  unsigned char *ringA = smem;                  // 2 x 32 KB
  unsigned char *ringB = smem + 2 * kAStage;    // 2 x 16 KB
  // outside the accumulation (ring idle): diagonal factor scratch, then TRSM operands
  float *S = reinterpret_cast<float *>(smem);              // [T][LDS]
  float *Di = S + T * LDS;                                 // [T][LDS]
  unsigned char *Ax = smem;                                // 128 x 64 hi (32 KB) + lo (32 KB)
  unsigned char *Binv = smem + 2 * kAStage;                // 64 x 64 hi (16 KB) + lo (16 KB)

  const int b = blist[blockIdx.x];
  const BlockDesc B = blk[b];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int I = tid; I < B.nt; I += kThreads) s_tr[I] = trow[B.trow0 + I];
  const TileRow *tr = s_tr;
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&ctl.full_a[s], 1);
      mbar_init(&ctl.empty_a[s], 1);
      mbar_init(&ctl.full_b[s], 1);
      mbar_init(&ctl.empty_b[s], 1);
    }
    mbar_init(&ctl.acc_ready, 1);
    mbar_init(&ctl.trsm_ready, kEpi);
    mbar_init(&ctl.trsm_done, 1);
    ctl.abort = 0;
    ctl.fail = 0;
    ctl.pmin = 1e300;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&ctl.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = ctl.tmem_base;

  // phase / stage counters (each role keeps its own copy of the ones it uses)
  uint32_t na = 0, nb = 0;              // A / B stages issued (producer) or consumed (MMA)
  uint32_t ph_acc = 0, ph_ready = 0, ph_done = 0;

  for (int K = 0; K < B.nt; ++K) {
    // panel rows, computed by every thread alike (tile rows are few)
    if (tid == 0) {
      int n = 0;
      for (int I = K; I < B.nt; ++I)
        if (tr[I].j0 <= K) s_rows[n++] = I;
      s_nrows = n;
    }
    __syncthreads();
    const int nrows = s_nrows;
    const int npairs = (nrows + 1) / 2;
    const int jlo = tr[K].j0;  // row K's envelope: L_KJ != 0 for jlo <= J < K
    for (int p0 = 0; p0 < npairs; p0 += kPairsMax) {
      const int np = min(kPairsMax, npairs - p0);
      // rows of pair p of this pass (I1 < 0: single tile)
      auto pair_rows = [&](int p, int &I0, int &I1) {
        I0 = s_rows[2 * (p0 + p)];
        I1 = 2 * (p0 + p) + 1 < nrows ? s_rows[2 * (p0 + p) + 1] : -1;
      };
      auto pair_has = [&](int I0, int I1, int J) {
        return tr[I0].j0 <= J || (I1 >= 0 && tr[I1].j0 <= J);
      };
      auto pass_has = [&](int J) {
        for (int p = 0; p < np; ++p) {
          int I0, I1;
          pair_rows(p, I0, I1);
          if (pair_has(I0, I1, J)) return true;
        }
        return false;
      };
      if (warp == 4) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
          for (int J = jlo; J < K; ++J) {
            if (!pass_has(J)) continue;
            for (int h = 0; h < 2; ++h) {
              const uint32_t sb = nb & 1;
              if (nb >= 2 && !wait_phase(&ctl, &ctl.empty_b[sb], ((nb >> 1) - 1) & 1, err)) break;
              if (ctl.abort) break;
              unsigned char *dst = ringB + sb * kBStage;
              const float *img = lc + 2 * tile_index(tr[K], J);
              mbar_expect_tx(&ctl.full_b[sb], kBStage);
              bulk_g2s(dst, img + h * (kHalf / 4), kHalf, &ctl.full_b[sb]);
              bulk_g2s(dst + kHalf, img + (2 + h) * (kHalf / 4), kHalf, &ctl.full_b[sb]);
              ++nb;
              for (int p = 0; p < np; ++p) {
                int I0, I1;
                pair_rows(p, I0, I1);
                if (!pair_has(I0, I1, J)) continue;
                const uint32_t sa = na & 1;
                if (na >= 2 && !wait_phase(&ctl, &ctl.empty_a[sa], ((na >> 1) - 1) & 1, err))
                  break;
                if (ctl.abort) break;
                unsigned char *da = ringA + sa * kAStage;
                const float *i0 = tr[I0].j0 <= J ? lc + 2 * tile_index(tr[I0], J) : nullptr;
                const float *i1 =
                    (I1 >= 0 && tr[I1].j0 <= J) ? lc + 2 * tile_index(tr[I1], J) : nullptr;
                mbar_expect_tx(&ctl.full_a[sa], kAStage);
                bulk_g2s(da, i0 ? i0 + h * (kHalf / 4) : zero_img, kHalf, &ctl.full_a[sa]);
                bulk_g2s(da + kHalf, i1 ? i1 + h * (kHalf / 4) : zero_img, kHalf,
                         &ctl.full_a[sa]);
                bulk_g2s(da + 2 * kHalf, i0 ? i0 + (2 + h) * (kHalf / 4) : zero_img, kHalf,
                         &ctl.full_a[sa]);
                bulk_g2s(da + 3 * kHalf, i1 ? i1 + (2 + h) * (kHalf / 4) : zero_img, kHalf,
                         &ctl.full_a[sa]);
                ++na;
              }
            }
          }
        }
      } else if (warp == 5) {
        // ---------------------------------------------------------------- MMA issue
        if (lane == 0) {
          uint32_t started = 0;  // bit p: pair p has its first product in this pass
          for (int J = jlo; J < K && !ctl.abort; ++J) {
            if (!pass_has(J)) continue;
            for (int h = 0; h < 2 && !ctl.abort; ++h) {
              const uint32_t sb = nb & 1;
              if (!wait_phase(&ctl, &ctl.full_b[sb], (nb >> 1) & 1, err)) break;
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              const uint32_t bh = smem_u32(ringB + sb * kBStage), bl = bh + kHalf;
              for (int p = 0; p < np; ++p) {
                int I0, I1;
                pair_rows(p, I0, I1);
                if (!pair_has(I0, I1, J)) continue;
                const uint32_t sa = na & 1;
                if (!wait_phase(&ctl, &ctl.full_a[sa], (na >> 1) & 1, err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ah = smem_u32(ringA + sa * kAStage), al = ah + 2 * kHalf;
                mma_3x(tmem + 64 * p, ah, al, bh, bl, 1024, 4, (started >> p) & 1u);
                started |= 1u << p;
                mma_commit(&ctl.empty_a[sa]);
                ++na;
              }
              mma_commit(&ctl.empty_b[sb]);
              ++nb;
            }
          }
          mma_commit(&ctl.acc_ready);
          // TRSM of every pair, once the epilogue has staged its operand
          for (int p = 0; p < np; ++p) {
            if (!wait_phase(&ctl, &ctl.trsm_ready, ph_ready & 1, err)) break;
            ++ph_ready;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = smem_u32(Ax), al = ah + 32768;
            const uint32_t bh = smem_u32(Binv), bl = bh + 16384;
            mma_3x(tmem + 64 * p, ah, al, bh, bl, 2048, 8, false);
            mma_commit(&ctl.trsm_done);
          }
        }
      } else {
        // ---------------------------------------------------------------- epilogue (0-3)
        const int t = tid;  // accumulator row
        // tcgen05.ld is warp-collective: every decision before one is made warp-uniform
        bool ok = __all_sync(0xffffffffu, wait_phase(&ctl, &ctl.acc_ready, ph_acc & 1, err));
        ++ph_acc;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        if (p0 == 0) {
          // diagonal tile: S = G_KK - D_K (rows 0..63 of pair 0)
          float d[64];
          int I0, I1;
          pair_rows(0, I0, I1);
          const bool acc0 = jlo < K;
          if (acc0 && ok) {
            tmem_ld64(tmem + lane_base, d);
          } else {
#pragma unroll
            for (int c = 0; c < 64; ++c) d[c] = 0.f;
          }
          if (t < T) {
            const float *g = fac + tile_index(tr[K], K) + t * T;
#pragma unroll
            for (int c = 0; c < T; c += 4) {
              const float4 x = *reinterpret_cast<const float4 *>(g + c);
              S[t * LDS + c] = c <= t ? x.x - d[c] : 0.f;
              S[t * LDS + c + 1] = c + 1 <= t ? x.y - d[c + 1] : 0.f;
              S[t * LDS + c + 2] = c + 2 <= t ? x.z - d[c + 2] : 0.f;
              S[t * LDS + c + 3] = c + 3 <= t ? x.w - d[c + 3] : 0.f;
            }
          }
          epi_sync();
          diag_factor_blocked(S, Di, Di + T * LDS, t, B.m - K * T, &ctl.pmin, &ctl.fail);
          float *gKK = fac + tile_index(tr[K], K);
          float *dK = dinv + B.dinv_off + (int64_t)K * T * T;
          for (int e = t; e < T * T; e += kEpi) {
            const int r = e / T, c = e % T;
            gKK[e] = c <= r ? S[r * LDS + c] : 0.f;
            dK[e] = c <= r ? Di[r * LDS + c] : 0.f;
          }
          epi_sync();  // S / Di are read; the TRSM operands may overwrite them
        }
        // B operand of the TRSM: rows of inv(L_KK) (B[n][k] = inv(L_KK)[n][k]), full K
        {
          const float *dK = dinv + B.dinv_off + (int64_t)K * T * T;
          for (int e = t; e < T * T; e += kEpi) {
            const int n = e / T, k = e % T;
            const float x = dK[e];
            const float hi = tf32_hi(x);
            *reinterpret_cast<float *>(Binv + full_off(n, k)) = hi;
            *reinterpret_cast<float *>(Binv + 16384 + full_off(n, k)) = x - hi;
          }
        }
        for (int p = 0; p < np; ++p) {
          int I0, I1;
          pair_rows(p, I0, I1);
          const int I = t < T ? I0 : I1;
          const bool real = I >= 0 && I != K;  // rows of this thread's tile to solve
          // X = G_IK - D_I, split into the A operand (rows of the pair, full K)
          const bool accp = ok && pair_has(I0, I1, jlo < K ? K - 1 : -1) && jlo < K;
          float d[64];
          if (accp) {
            tmem_ld64(tmem + lane_base + 64 * p, d);
          } else {
#pragma unroll
            for (int c = 0; c < 64; ++c) d[c] = 0.f;
          }
          const float *g = real ? fac + tile_index(tr[I], K) + (t & 63) * T : nullptr;
#pragma unroll
          for (int c = 0; c < 64; c += 4) {
            float4 x = real ? *reinterpret_cast<const float4 *>(g + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            x.x -= d[c];
            x.y -= d[c + 1];
            x.z -= d[c + 2];
            x.w -= d[c + 3];
            if (!real) x = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
            *reinterpret_cast<float4 *>(Ax + full_off(t, c)) = h;
            *reinterpret_cast<float4 *>(Ax + 32768 + full_off(t, c)) =
                make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(&ctl.trsm_ready);
          ok = __all_sync(0xffffffffu, ok && wait_phase(&ctl, &ctl.trsm_done, ph_done & 1, err));
          ++ph_done;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          float l[64];
          if (ok) {
            tmem_ld64(tmem + lane_base + 64 * p, l);
          } else {
#pragma unroll
            for (int c = 0; c < 64; ++c) l[c] = 0.f;
          }
          if (real && ok) {
            const int r = t & 63;
            float *o = fac + tile_index(tr[I], K) + r * T;
            float *img = lc + 2 * tile_index(tr[I], K);
#pragma unroll
            for (int c = 0; c < 64; c += 4) {
              const float4 v = make_float4(l[c], l[c + 1], l[c + 2], l[c + 3]);
              *reinterpret_cast<float4 *>(o + c) = v;
              const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
              // hi at K-half images 0 / 1, lo at 2 / 3
              *reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(img) + half_off(r, c)) = h;
              *reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(img) + 2 * kHalf +
                                          half_off(r, c)) =
                  make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
            }
          }
        }
        // the finished tiles are read by the next passes' bulk copies (async proxy)
        asm volatile("fence.proxy.async.global;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      }
      // end of the pass: the next one reads what this one wrote, and reuses tensor memory
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
  }
  // Without an abort every copy the producer issued was waited for by the MMA thread.  After
  // an abort the producer waits (bounded) for the last copy into each of its slots.
  if (warp == 4 && lane == 0 && ctl.abort) {
    auto drain = [&](uint64_t *full, uint32_t n) {
      for (uint32_t s = 0; s < 2 && s < n; ++s) {
        const uint32_t last = n - 1 - ((n - 1 - s) & 1);  // last use of slot s
        const uint64_t t0 = global_ns();
        while (!mbar_try_wait(&full[s], (last >> 1) & 1) && global_ns() - t0 < kWaitNs) {
        }
      }
    };
    drain(ctl.full_a, na);
    drain(ctl.full_b, nb);
  }
  __syncthreads();
  if (tid == 0) {
    pivmin[b] = ctl.pmin;
    pivfail[b] = ctl.fail | ctl.abort;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

// N_KJ = inv(L_KK) L_KJ in place for every off-diagonal tile of row K (CUDA cores, FP32):
// one CTA per tile row, 16 x 16 threads with 4 x 4 register tiles; inv(L_KK) is lower
// triangular, so row block R of the output needs k < 16 (R + 1).
__global__ void __launch_bounds__(256)
    k_ntransform(const BlockDesc *__restrict__ blk, const int32_t *__restrict__ rowblk_t,
                 const TileRow *__restrict__ trow, float *__restrict__ fac,
                 const float *__restrict__ dinv) {
  __shared__ __align__(16) float Di[T][T + 4];  // Di[r][k]
  __shared__ __align__(16) float L[T][T + 4];   // L[k][c]
  const int row = blockIdx.x;                   // global tile row
  const int b = rowblk_t[row];
  const BlockDesc B = blk[b];
  const int K = row - B.trow0;
  const TileRow TK = trow[row];
  if (TK.j0 >= K) return;
  const int tid = threadIdx.x, tr4 = tid >> 4, tc4 = tid & 15;
  const float *dK = dinv + B.dinv_off + (int64_t)K * T * T;
  for (int e = tid; e < T * T; e += 256) Di[e / T][e % T] = dK[e];
  for (int J = TK.j0; J < K; ++J) {
    float *g = fac + TK.off + (int64_t)(J - TK.j0) * T * T;
    __syncthreads();
    for (int e = tid; e < T * T / 4; e += 256) {
      const int k = e / (T / 4), c = 4 * (e % (T / 4));
      *reinterpret_cast<float4 *>(&L[k][c]) = *reinterpret_cast<const float4 *>(g + k * T + c);
    }
    __syncthreads();
    float acc[4][4] = {};
    const int kend = 4 * tr4 + 4;  // k <= the thread's last row
    for (int k = 0; k < kend; ++k) {
      const float4 lv = *reinterpret_cast<const float4 *>(&L[k][4 * tc4]);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float a = Di[4 * tr4 + i][k];
        acc[i][0] = fmaf(a, lv.x, acc[i][0]);
        acc[i][1] = fmaf(a, lv.y, acc[i][1]);
        acc[i][2] = fmaf(a, lv.z, acc[i][2]);
        acc[i][3] = fmaf(a, lv.w, acc[i][3]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      *reinterpret_cast<float4 *>(g + (4 * tr4 + i) * T + 4 * tc4) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
  }
}

__global__ void k_tile_row_blocks(const BlockDesc *__restrict__ blk, int32_t nblk,
                                  int32_t *__restrict__ rowblk_t) {
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const BlockDesc B = blk[b];
  for (int I = threadIdx.x; I < B.nt; I += blockDim.x) rowblk_t[B.trow0 + I] = b;
}

constexpr int kTcSmem = (int)kRing;
static_assert((2 * T * LDS + 3 * 256) * 4 <= 2 * kAStage, "diagonal scratch inside the A stages");

}  // namespace

int64_t cholesky_tc_scratch_floats(int64_t factor_elems) { return 2 * factor_elems + kHalf / 4; }

void launch_cholesky_tc(const BlockDesc *blk, const int32_t *blist, int32_t nlist, int32_t nblk,
                        int32_t ntrow, const TileRow *trow, float *fac, float *dinv,
                        float *scratch, int64_t factor_elems, int32_t *rowblk_t, double *pivmin,
                        int32_t *pivfail, int32_t *err, cudaStream_t s) {
  if (nlist <= 0) return;
  float *zero_img = scratch + 2 * factor_elems;
  cudaMemsetAsync(zero_img, 0, kHalf, s);
  cudaFuncSetAttribute(k_cholesky_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  k_cholesky_tc<<<(unsigned)nlist, kThreads, kTcSmem, s>>>(blk, blist, trow, fac, dinv, scratch,
                                                           zero_img, pivmin, pivfail, err);
}

void launch_ntransform_tc(const BlockDesc *blk, int32_t nblk, int32_t ntrow, const TileRow *trow,
                          float *fac, const float *dinv, int32_t *rowblk_t, cudaStream_t s) {
  if (nblk <= 0) return;
  k_tile_row_blocks<<<(unsigned)nblk, 64, 0, s>>>(blk, nblk, rowblk_t);
  k_ntransform<<<(unsigned)ntrow, 256, 0, s>>>(blk, rowblk_t, trow, fac, dinv);
}

}  // namespace cimmino
