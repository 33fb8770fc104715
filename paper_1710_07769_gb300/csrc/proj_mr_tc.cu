// Multi-right-hand-side projection on the tensor cores: the inner solves of Algorithm 2
// step 5 for a group of 16 CG lanes that share the FP32 factors of block i,
//   Y_i = G_i^{-1} U_i = L^{-T} L^{-1} U_i,   L = diag(L_II)(I + N),
// with every tile product an M = 128, N = 16 MMA (tcgen05, kind::tf32, 3xTF32 split:
// x = hi + lo, hi = x rounded to TF32, lo = (x - hi) rounded to TF32;
// A B = A_hi B_hi + A_hi B_lo + A_lo B_hi).
//
// W (the block's 16 columns) stays in tensor memory for the whole solve: tile rows 2p and
// 2p + 1 form the 128 x 16 FP32 accumulator of pair p (row t of the pair at lane t, right-
// hand side g at column 16 p + g), so a block of up to 32 tile rows takes 256 columns and
// two blocks share an SM.  An MMA's A operand is two 64 x 64 operator tiles stacked (the
// two rows of a pair), loaded by TMA with the 128-byte swizzle; a row of the pair that takes
// no part gets a zero tile (the copy starts at a negative row: the tensor map fills zeros).
// Its B operand is the 64 x 16 image of one tile row of W.  The four phases:
//   F0  W_I = inv(L_II) W_I for every I   (A = [inv(L_2p,2p); 0], then [0; inv(L_2p+1,2p+1)])
//   F1  J ascending: once W_J is final, W_I -= N_IJ W_J for every I > J in the envelope
//       (right-looking: W_J's image is made once and feeds all pairs below it)
//   B1  J descending: W_I -= NT_IJ W_J for I < J  (NT_IJ = N_JI^T, the transposed copy)
//   B2  W_I = inv(L_II)^T W_I
// F1 and B1 subtract by using the negated image of W_J.
//
// Roles (320 threads): warps 0-3 (E) move tile rows of W from tensor memory into B images
// (hi/lo split, 128-byte swizzle) and wait for the accumulators; warps 4-7 (C) split every
// operator image that TMA has landed into its hi and lo parts in place; warp 8 (one lane)
// issues the MMAs; warp 9 (one lane) issues the TMA loads.  E and C together put U into
// tensor memory, add W into y (FP64) and, for FP32 refinement, compute the residual
// u - G_i y in FP64 from the sliced-ELL Gram copy, which becomes the next pass's right-hand
// side in tensor memory; the steps stop once every active lane has ||res|| <= tol ||u||.
// The order of all operator tiles, MMAs and images of a pass is one list of work units
// (K-half of one pair product) built once per block; the roles walk it in step.
// Every wait is bounded by %globaltimer: after about 2 s the kernel sets bit 16 of the
// error word and every later wait returns at once, so the kernel always ends.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace cimmino {

namespace {

constexpr int T = kTile;
constexpr int64_t TT = (int64_t)T * T;
constexpr int RG = 16;                     // right-hand sides per group = MMA N
constexpr int kMaxNt = 32;                 // tile rows: 16 pairs x 16 columns of TMEM
constexpr int kThreads = 320;
constexpr int kWork = 256;                 // warps 0-7 (E and C)
constexpr int kASlots = 2;
constexpr uint32_t kAHalf = 16384;         // one K-half of a pair: 128 rows x 128 B
constexpr uint32_t kASlot = 2 * kAHalf;    // hi (the TMA image, split in place), lo
constexpr int kBSlots = 3;
constexpr uint32_t kBImg = 4096;           // 16 rows x 64 columns x 4 B
constexpr uint32_t kBSlot = 2 * kBImg;     // hi, lo
constexpr int kDynSmem = 1024 + kASlots * kASlot + kBSlots * kBSlot;
// units per pass at most: F0 and B2 4 per pair, F1 and B1 2 per (step, pair) in the triangle
constexpr int kMaxUnits = 2 * 64 + 2 * 512;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int32_t kErrBit = 16;
// D f32, A/B tf32, both K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) |
                            ((128u >> 4) << 24);

// ---- a work unit: K-half h of the product of pair p with one image, as a 32-bit word
//   bits 0-3 p | 4 h | 5 image of the group (F0/B2: 0 = tile 2p, 1 = tile 2p + 1)
//   6-7 phase (0 F0, 1 F1, 2 B1, 3 B2) | 8 top tile present | 9 bottom tile present
//   10-14 J (F1/B1 step) | 15 first product of the pair (overwrites the accumulator)
//   16-17 images to wait for first | 18-19 images released after it
//   20 accumulators committed before it | 21 committed after it
constexpr uint32_t U_TOP = 1u << 8, U_BOT = 1u << 9, U_FIRST = 1u << 15;
constexpr uint32_t U_ACC_BEFORE = 1u << 20, U_ACC_AFTER = 1u << 21;
__device__ __forceinline__ uint32_t unit_word(int p, int h, int sub, int phase, bool top,
                                              bool bot, int J) {
  return (uint32_t)p | ((uint32_t)h << 4) | ((uint32_t)sub << 5) | ((uint32_t)phase << 6) |
         (top ? U_TOP : 0u) | (bot ? U_BOT : 0u) | ((uint32_t)J << 10);
}
__device__ __forceinline__ uint32_t u_wait(int n) { return (uint32_t)n << 16; }
__device__ __forceinline__ uint32_t u_rel(int n) { return (uint32_t)n << 18; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
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
  uint64_t raw[kASlots];      // TMA image landed
  uint64_t a_full[kASlots];   // hi/lo split done (4 C warps)
  uint64_t a_empty[kASlots];  // MMAs of the slot done
  uint64_t b_full[kBSlots];   // image written (4 E warps)
  uint64_t b_empty[kBSlots];  // MMAs reading the image done
  uint64_t acc;               // accumulators ready for E
  uint64_t fin;               // every MMA done (before tensor memory is freed)
  uint32_t tmem;
  int abort;
};

// Bounded wait on a barrier phase; gives up (and makes every later wait give up) after about
// 2 s or once another role has given up.
__device__ __forceinline__ bool wait_bar(Ctl &c, uint64_t *b, uint32_t parity, int32_t *err) {
  if (*(volatile int *)&c.abort) return false;
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < (1u << 30); ++i) {
    if (mbar_try_wait(b, parity)) return true;
    if (*(volatile int *)&c.abort) return false;
    if (global_ns() - t0 > kWaitNs) break;
  }
  *(volatile int *)&c.abort = 1;
  atomicOr(err, kErrBit);
  return false;
}

// K-major operand with the 128-byte swizzle: rows of 128 B (32 TF32 values), 8-row groups
// 1024 B apart; a K step of 8 advances the start by 32 B inside the swizzle atom
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return __uint_as_float(h);
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
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// 64 rows x 32 columns of the [rows][64] FP32 view `tm`, starting at (x, y)
__device__ __forceinline__ void tma_box(void *dst, const CUtensorMap *tm, int x, int y,
                                        uint64_t *bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(tm), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15,%16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
      : "memory");
}
__device__ __forceinline__ void work_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// per right-hand side sum over the 256 work threads in a fixed order: warp sums, then the
// 8 warps in order; result in out[0..15] (tmp: 8 x 16 doubles)
__device__ __forceinline__ void work_sum16(const double (&v)[RG], double *tmp, double *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < RG; ++g) {
    const double s = warp_sum(v[g]);
    if (lane == 0) tmp[warp * RG + g] = s;
  }
  work_sync();
  if (threadIdx.x < RG) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += tmp[w * RG + threadIdx.x];
    out[threadIdx.x] = s;
  }
  work_sync();
}

// the same for 8 right-hand sides
__device__ __forceinline__ void work_sum8(const double (&v)[8], double *tmp, double *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const double s = warp_sum(v[g]);
    if (lane == 0) tmp[warp * 8 + g] = s;
  }
  work_sync();
  if (threadIdx.x < 8) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += tmp[w * 8 + threadIdx.x];
    out[threadIdx.x] = s;
  }
  work_sync();
}

__global__ void __launch_bounds__(kThreads, 2)
    k_proj_mr_tc(const IterArgs a, const __grid_constant__ CUtensorMap tm_fac,
                 const __grid_constant__ CUtensorMap tm_facT,
                 const __grid_constant__ CUtensorMap tm_dinv,
                 const __grid_constant__ CUtensorMap tm_dinvT, const double *__restrict__ u,
                 double *__restrict__ y, int check_lane) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ Ctl ctl;
  __shared__ TileRow s_tr[kMaxNt], s_trT[kMaxNt];
  __shared__ uint32_t s_f1[kMaxNt], s_b1[kMaxNt];  // pairs updated by step J (bit p)
  __shared__ int s_off1[kMaxNt], s_off2[kMaxNt], s_nunits;
  __shared__ uint32_t s_units[kMaxUnits];
  __shared__ double s_tmp[8 * RG], s_un2[RG], s_e2[RG];
  __shared__ int s_again;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const BlockDesc B = a.blk[a.mr_list[blockIdx.x]];
  const int nt = B.nt, npairs = (nt + 1) >> 1;
  unsigned char *base = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
  unsigned char *aslot = base;                      // kASlots x (hi, lo)
  unsigned char *bslot = base + kASlots * kASlot;   // kBSlots x (hi, lo)

  for (int I = tid; I < nt; I += kThreads) {
    s_tr[I] = a.trow[B.trow0 + I];
    s_trT[I] = a.trowT[B.trow0 + I];
  }
  if (tid == 0) {
    for (int s = 0; s < kASlots; ++s) {
      mbar_init(&ctl.raw[s], 1);
      mbar_init(&ctl.a_full[s], 4);
      mbar_init(&ctl.a_empty[s], 1);
    }
    for (int s = 0; s < kBSlots; ++s) {
      mbar_init(&ctl.b_full[s], 4);
      mbar_init(&ctl.b_empty[s], 1);
    }
    mbar_init(&ctl.acc, 1);
    mbar_init(&ctl.fin, 1);
    ctl.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const uint32_t ncols = npairs <= 2 ? 32u : npairs <= 4 ? 64u : npairs <= 8 ? 128u : 256u;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&ctl.tmem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = ctl.tmem;

  // ---- the unit list of one pass (the same for every pass and group of this block)
  if (tid < nt) {
    const int J = tid;
    uint32_t f = 0, bm = 0;
    for (int I = J + 1; I < nt; ++I)
      if (s_tr[I].j0 <= J) f |= 1u << (I >> 1);
    for (int I = s_tr[J].j0; I < J; ++I) bm |= 1u << (I >> 1);
    s_f1[J] = f;
    s_b1[J] = bm;
  }
  __syncthreads();
  const int nf0 = 4 * npairs - ((nt & 1) ? 2 : 0);
  if (tid == 0) {
    int o = nf0;
    for (int J = 0; J < nt; ++J) {
      s_off1[J] = o;
      o += 2 * __popc(s_f1[J]);
    }
    for (int J = nt - 1; J >= 0; --J) {
      s_off2[J] = o;
      o += 2 * __popc(s_b1[J]);
    }
    s_nunits = o + nf0;
  }
  __syncthreads();
  const int nunits = s_nunits;
  if (tid < npairs) {
    // F0 (units [0, nf0)) and B2 (the last nf0 units): per pair (tile 2p, h0), (2p+1, h0),
    // (2p, h1), (2p+1, h1), so that the two A slots keep the zero half in the same place
    const int p = tid;
    const bool two = 2 * p + 1 < nt;
    for (int ph = 0; ph < 2; ++ph) {
      const int phase = ph == 0 ? 0 : 3;
      uint32_t *o = s_units + (ph == 0 ? 0 : nunits - nf0) + 4 * p;
      if (two) {
        o[0] = unit_word(p, 0, 0, phase, true, false, 0) | U_FIRST | u_wait(2);
        o[1] = unit_word(p, 0, 1, phase, false, true, 0);
        o[2] = unit_word(p, 1, 0, phase, true, false, 0) | u_rel(1);
        o[3] = unit_word(p, 1, 1, phase, false, true, 0) | u_rel(1);
        if (p == npairs - 1) o[3] |= U_ACC_AFTER;
      } else {
        o[0] = unit_word(p, 0, 0, phase, true, false, 0) | U_FIRST | u_wait(1);
        o[1] = unit_word(p, 1, 0, phase, true, false, 0) | u_rel(1) | U_ACC_AFTER;
      }
    }
  }
  if (tid < nt) {
    const int J = tid;
    // F1 step J: pairs with a row I > J inside the envelope; the pair holding the next
    // step's row goes first and the accumulators are committed right after it
    for (int sweep = 0; sweep < 2; ++sweep) {
      const uint32_t M = sweep == 0 ? s_f1[J] : s_b1[J];
      if (!M) continue;
      int Jn = -1;
      if (sweep == 0) {
        for (int K = J + 1; K < nt; ++K)
          if (s_f1[K]) { Jn = K; break; }
      } else {
        for (int K = J - 1; K >= 0; --K)
          if (s_b1[K]) { Jn = K; break; }
      }
      const int cp = Jn >= 0 ? (Jn >> 1) : -1;
      const bool crit = cp >= 0 && ((M >> cp) & 1u);
      uint32_t *o = s_units + (sweep == 0 ? s_off1[J] : s_off2[J]);
      int n = 0;
      auto emit = [&](int p) {
        const int I0 = 2 * p, I1 = 2 * p + 1;
        bool top, bot;
        if (sweep == 0) {
          top = I0 > J && s_tr[I0].j0 <= J;
          bot = I1 < nt && I1 > J && s_tr[I1].j0 <= J;
        } else {
          top = I0 < J && I0 >= s_tr[J].j0;
          bot = I1 < J && I1 >= s_tr[J].j0;
        }
        for (int h = 0; h < 2; ++h) o[n++] = unit_word(p, h, 0, 1 + sweep, top, bot, J);
      };
      if (crit) emit(cp);
      for (uint32_t r = M; r; r &= r - 1) {
        const int p = __ffs(r) - 1;
        if (!(crit && p == cp)) emit(p);
      }
      o[0] |= u_wait(1);
      o[n - 1] |= u_rel(1);
      if (Jn < 0)
        o[n - 1] |= U_ACC_AFTER;
      else if (crit)
        o[1] |= U_ACC_AFTER;
      else
        o[0] |= U_ACC_BEFORE;
    }
  }
  __syncthreads();

  // role counters, kept across passes and groups
  uint32_t n_tma = 0, n_split = 0, n_mma = 0, n_bw = 0, n_br = 0, n_img = 0, n_acc = 0;
  const uint64_t policy = l2_evict_first();
  const bool work = tid < kWork;
  const int q = warp & 3, wh = (warp >> 2) & 1;  // TMEM quadrant; E (0) or C (1) half
  const int64_t ld = a.nrhs;
  const int refine_steps = a.refine_steps;

  for (int k0 = 0; k0 < a.nrhs; k0 += RG) {
    const int ng = min(RG, a.nrhs - k0);
    uint32_t mask = 0;
    for (int g = 0; g < ng; ++g)
      if (!check_lane || a.lane[B.sys * a.nrhs + k0 + g].status == CIMMINO_RUNNING)
        mask |= 1u << g;
    if (!mask) continue;
    // U (rows of this thread's pairs) into tensor memory
    if (work) {
      double un2[RG];
#pragma unroll
      for (int g = 0; g < RG; ++g) un2[g] = 0.0;
      for (int p = wh; p < npairs; p += 2) {
        const int r = 128 * p + 32 * q + lane;
        float v[RG];
        const double *ur = u + (B.row0 + r) * ld + k0;
#pragma unroll
        for (int g = 0; g < RG; ++g) {
          const double x = (r < B.m && ((mask >> g) & 1u)) ? ur[g] : 0.0;
          v[g] = (float)x;
          un2[g] += x * x;
        }
        tmem_st16(tmem + ((uint32_t)(32 * q) << 16) + 16 * p, v);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      if (refine_steps > 0) work_sum16(un2, s_tmp, s_un2);
    }
    int s = 0;
    for (;;) {
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (warp == 9) {
        // -------------------------------------------------------------- TMA producer
        if (lane == 0) {
          // the operator boxes of unit i: map and rows of the top and bottom tiles (-T: none)
          auto source = [&](uint32_t w, const CUtensorMap *&tm, int &yt, int &yb) {
            const int ph = (w >> 6) & 3, p = w & 15, J = (w >> 10) & 31;
            tm = ph == 0 ? &tm_dinv : ph == 1 ? &tm_fac : ph == 2 ? &tm_facT : &tm_dinvT;
            auto row_of = [&](int I) -> int {
              int64_t e;
              if (ph == 1)
                e = s_tr[I].off + (int64_t)(J - s_tr[I].j0) * TT;
              else if (ph == 2)
                e = s_trT[I].off + (int64_t)(J - I - 1) * TT;
              else
                e = B.dinv_off + (int64_t)I * TT;
              return (int)(e >> 6);
            };
            yt = (w & U_TOP) ? row_of(2 * p) : -T;
            yb = (w & U_BOT) ? row_of(2 * p + 1) : -T;
          };
          for (int i = 0; i < nunits; ++i) {
            const uint32_t w = s_units[i];
            const uint32_t sl = n_tma % kASlots;
            if (n_tma >= kASlots &&
                !wait_bar(ctl, &ctl.a_empty[sl], ((n_tma / kASlots) - 1) & 1, a.err))
              break;
            const CUtensorMap *tm;
            int yt, yb;
            source(w, tm, yt, yb);
            const int h = (w >> 4) & 1;
            unsigned char *dst = aslot + sl * kASlot;
            mbar_expect_tx(&ctl.raw[sl], kAHalf);
            tma_box(dst, tm, 32 * h, yt, &ctl.raw[sl], policy);
            tma_box(dst + kAHalf / 2, tm, 32 * h, yb, &ctl.raw[sl], policy);
            ++n_tma;
          }
        }
      } else if (warp == 8) {
        // -------------------------------------------------------------- MMA issue
        if (lane == 0) {
          uint32_t grp = 0;  // first image of the current group
          for (int i = 0; i < nunits; ++i) {
            const uint32_t w = s_units[i];
            const int nw = (w >> 16) & 3;
            bool ok = true;
            if (nw) {
              grp = n_bw;
              for (int k = 0; k < nw; ++k, ++n_bw)
                ok = ok && wait_bar(ctl, &ctl.b_full[n_bw % kBSlots], (n_bw / kBSlots) & 1, a.err);
            }
            // a commit before the step's products is still issued after its image has
            // arrived: E made that image after taking the previous commit, so at most one
            // phase of `acc` is ever outstanding
            if (w & U_ACC_BEFORE) mma_commit(&ctl.acc);
            const uint32_t sl = n_mma % kASlots;
            ok = ok && wait_bar(ctl, &ctl.a_full[sl], (n_mma / kASlots) & 1, a.err);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t img = grp + ((w >> 5) & 1);
            const uint32_t bh = smem_u32(bslot + (img % kBSlots) * kBSlot), bl = bh + kBImg;
            const uint32_t ah = smem_u32(aslot + sl * kASlot), al = ah + kAHalf;
            const int p = w & 15, h = (w >> 4) & 1;
            const bool first = (w & U_FIRST) != 0;
            const uint32_t d = tmem + 16 * p;
#pragma unroll
            for (int st = 0; st < 4; ++st) {
              const uint32_t ao = 32 * st, bo = 2048 * h + 32 * st;
              mma_tf32(d, desc_sw128(ah + ao), desc_sw128(bh + bo), !(first && st == 0));
              mma_tf32(d, desc_sw128(ah + ao), desc_sw128(bl + bo), 1);
              mma_tf32(d, desc_sw128(al + ao), desc_sw128(bh + bo), 1);
            }
            mma_commit(&ctl.a_empty[sl]);
            ++n_mma;
            const int nr = (w >> 18) & 3;
            for (int k = 0; k < nr; ++k, ++n_br) mma_commit(&ctl.b_empty[n_br % kBSlots]);
            if (w & U_ACC_AFTER) mma_commit(&ctl.acc);
          }
        }
      } else if (warp >= 4) {
        // -------------------------------------------------------------- hi/lo split (C)
        const int ct = tid - 128;
        for (int i = 0; i < nunits; ++i) {
          const uint32_t sl = n_split % kASlots;
          const bool ok = wait_bar(ctl, &ctl.raw[sl], (n_split / kASlots) & 1, a.err);
          if (!__all_sync(0xffffffffu, ok)) break;
          float4 *hi = reinterpret_cast<float4 *>(aslot + sl * kASlot);
          float4 *lo = reinterpret_cast<float4 *>(aslot + sl * kASlot + kAHalf);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int e = ct + 128 * k;
            const float4 x = hi[e];
            const float4 hh = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
            hi[e] = hh;
            lo[e] = make_float4(tf32_hi(x.x - hh.x), tf32_hi(x.y - hh.y), tf32_hi(x.z - hh.z),
                                tf32_hi(x.w - hh.w));
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&ctl.a_full[sl]);
          ++n_split;
        }
      } else {
        // -------------------------------------------------------------- W -> B images (E)
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        // image k of tile row (2p + (q >> 1)) from this warp's 32 rows of pair p
        auto write_img = [&](uint32_t k, int p, bool neg) {
          float v[RG];
          tmem_ld16(tmem + lane_base + 16 * p, v);
          unsigned char *im = bslot + (k % kBSlots) * kBSlot + (q & 1) * 2048;
#pragma unroll
          for (int n = 0; n < RG; ++n) {
            const float x = neg ? -v[n] : v[n];
            const float hh = tf32_hi(x);
            const uint32_t off = n * 128 + ((((lane >> 2) ^ n) & 7) << 4) + (lane & 3) * 4;
            *reinterpret_cast<float *>(im + off) = hh;
            *reinterpret_cast<float *>(im + kBImg + off) = tf32_hi(x - hh);
          }
        };
        auto img_free = [&](uint32_t k) {
          return k < (uint32_t)kBSlots ||
                 wait_bar(ctl, &ctl.b_empty[k % kBSlots], ((k / kBSlots) - 1) & 1, a.err);
        };
        auto publish = [&](uint32_t k, int nimg) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0)
            for (int i = 0; i < nimg; ++i) mbar_arrive(&ctl.b_full[(k + i) % kBSlots]);
        };
        auto acc_wait = [&]() {
          const bool ok = __all_sync(0xffffffffu, wait_bar(ctl, &ctl.acc, n_acc & 1, a.err));
          ++n_acc;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          return ok;
        };
        // F0 / B2: both tiles of every pair
        auto diag_images = [&]() {
          for (int p = 0; p < npairs; ++p) {
            const int nimg = 2 * p + 1 < nt ? 2 : 1;
            const uint32_t k = n_img;
            n_img += nimg;
            bool ok = img_free(k);
            if (nimg == 2) ok = img_free(k + 1) && ok;
            ok = __all_sync(0xffffffffu, ok);
            if (ok && (q >> 1) < nimg) write_img(k + (q >> 1), p, false);
            publish(k, nimg);
          }
        };
        // F1 / B1 step J: the negated image of tile row J
        auto step_image = [&](int J) {
          bool ok = acc_wait();
          const uint32_t k = n_img++;
          ok = __all_sync(0xffffffffu, ok && img_free(k));
          if (ok && (q >> 1) == (J & 1)) write_img(k, J >> 1, true);
          publish(k, 1);
        };
        diag_images();
        for (int J = 0; J < nt; ++J)
          if (s_f1[J]) step_image(J);
        for (int J = nt - 1; J >= 0; --J)
          if (s_b1[J]) step_image(J);
        acc_wait();
        diag_images();
        acc_wait();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // y (+)= W
      if (work) {
        for (int p = wh; p < npairs; p += 2) {
          const int r = 128 * p + 32 * q + lane;
          float v[RG];
          tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + 16 * p, v);
          if (r < B.m) {
            double *yr = y + (B.row0 + r) * ld + k0;
#pragma unroll
            for (int g = 0; g < RG; ++g)
              if ((mask >> g) & 1u) yr[g] = s == 0 ? (double)v[g] : yr[g] + (double)v[g];
          }
        }
      }
      __syncthreads();
      int again = 0;
      if (s < refine_steps) {
        // res = u - G_i y into tensor memory; a warp covers whole 32-row slices of the Gram
        // copy; two sweeps of 8 right-hand sides each keep the FP64 accumulators in registers
        if (work) {
          for (int hg = 0; hg < 2; ++hg) {
            const int kg = k0 + 8 * hg;
            const uint32_t mh = (mask >> (8 * hg)) & 0xffu;
            double e2[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) e2[g] = 0.0;
            for (int p = wh; p < npairs; p += 2) {
              const int r = 128 * p + 32 * q + lane;
              float v[8];
              if (r < B.m && mh) {
                double acc[8];
                const double *ur = u + (B.row0 + r) * ld + kg;
#pragma unroll
                for (int g = 0; g < 8; ++g) acc[g] = ((mh >> g) & 1u) ? ur[g] : 0.0;
                gram_row_residual<8>(a, B, r, y, ld, kg, mh, acc);
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                  v[g] = (float)acc[g];
                  e2[g] += acc[g] * acc[g];
                }
              } else {
#pragma unroll
                for (int g = 0; g < 8; ++g) v[g] = 0.f;
              }
              tmem_st8(tmem + ((uint32_t)(32 * q) << 16) + 16 * p + 8 * hg, v);
            }
            work_sum8(e2, s_tmp, s_e2 + 8 * hg);
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          for (int g = 0; g < RG; ++g) {
            if (!((mask >> g) & 1u)) continue;
            const double tol = inner_tol(a, check_lane, (int64_t)B.sys * a.nrhs + k0 + g);
            if (s_e2[g] > tol * tol * s_un2[g]) again = 1;
          }
        }
      }
      if (tid == 0) s_again = again;
      __syncthreads();
      if (!s_again || *(volatile int *)&ctl.abort) break;
      ++s;
    }
    if (tid == 0 && refine_steps > 0) {
      atomicAdd(reinterpret_cast<unsigned long long *>(a.refine_total),
                (unsigned long long)s * (unsigned long long)__popc(mask));
      atomicMax(a.refine_max, s);
    }
  }
  // Without an abort every copy and MMA was waited for.  After one, the producer waits
  // (bounded) for the last copy into each slot and the MMA lane for its last MMAs.
  if (warp == 9 && lane == 0 && ctl.abort) {
    for (uint32_t sl = 0; sl < (uint32_t)kASlots && sl < n_tma; ++sl) {
      const uint32_t last = n_tma - 1 - ((n_tma - 1 - sl) % kASlots);
      const uint64_t t0 = global_ns();
      while (!mbar_try_wait(&ctl.raw[sl], (last / kASlots) & 1) && global_ns() - t0 < kWaitNs) {
      }
    }
  }
  if (warp == 8 && lane == 0) {
    mma_commit(&ctl.fin);
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(&ctl.fin, 0) && global_ns() - t0 < kWaitNs) {
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
}

}  // namespace

int proj_mr_tc_max_tiles() { return kMaxNt; }

// [rows][64] FP32 view of a tile array (64 x 64 tiles, row-major), loaded in boxes of 64 rows x
// 32 columns with the 128-byte swizzle; rows outside the array read as zeros.
bool make_tile_map(void *map, const float *base, int64_t elems) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const int64_t rows = elems / T;
  if (!base || rows < 1 || rows > (int64_t)INT32_MAX) return false;
  cuuint64_t dims[2] = {(cuuint64_t)T, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)T * sizeof(float)};
  cuuint32_t box[2] = {32, (cuuint32_t)T};
  cuuint32_t es[2] = {1, 1};
  return encode(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                const_cast<float *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t tile_map_bytes() { return sizeof(CUtensorMap); }

cudaError_t set_proj_mr_tc_smem_attr() {
  return cudaFuncSetAttribute(k_proj_mr_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kDynSmem);
}

void launch_proj_mr_tc(const IterArgs &a, const double *u, double *y, int check_lane,
                       cudaStream_t s) {
  const CUtensorMap *tm = static_cast<const CUtensorMap *>(a.mr_tmaps);
  k_proj_mr_tc<<<(unsigned)a.mr_ntc, kThreads, kDynSmem, s>>>(a, tm[0], tm[1], tm[2], tm[3], u,
                                                               y, check_lane);
}

}  // namespace cimmino
