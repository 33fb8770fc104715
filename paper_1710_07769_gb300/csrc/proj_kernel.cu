// Projection kernel: y_i = G_i^{-1} u_i for every block i (the inner solves of
// Algorithm 2 step 5, with G_i = A_i A_i^T = L_i L_i^T), one CTA per block.
//
// The factor is stored as L = diag(L_II) (I + N) with N_IJ = inv(L_II) L_IJ, together
// with inv(L_II) and transposed copies NT_IJ = N_JI^T, inv(L_II)^T.  Then
//   L z = b    <=>  c_I = inv(L_II) b_I (all I),  z_I = c_I - sum_{J<I} N_IJ z_J
//   L^T y = z  <=>  v_I = z_I - sum_{J>I} NT_IJ v_J,     y_I = inv(L_II)^T v_I (all I)
// so all four phases are row products of 64 x 64 tiles with a vector, and the two
// sequential chains (one step per tile row) need one reduction and one barrier per step.
//
// CTA = 8 consumer warps + 1 producer warp.
//  * The producer streams the tiles (16 or 32 KB) with cp.async.bulk into a ring of
//    shared-memory slots in the consumers' order.  full[s] completes when a copy lands,
//    empty[s] when all 8 consumer warps have passed the slot.  Every wait is bounded; a
//    wait that runs out sets the error flag and the kernel finishes without waiting again.
//  * inv(L_II) and its transpose (independent tile rows): one warp computes a tile, a lane
//    per row pair (p, 63 - p), no reduction.  They are streamed as packed triangles:
//    rectangular full packed in FP64 (2176 of 4096 values), block-packed in FP32 (2688).
//    Every consumer warp waits for and releases every slot in order, so a warp never waits on a slot more than one use ahead (which would
//    make the mbarrier phase parity ambiguous).
//  * Chain steps: every consumer thread does 16 FMAs per tile.  FP32: thread (rg, cg) owns
//    rows 4rg..4rg+3 and four columns (4 x 4 register block, 4 16-byte loads of the tile
//    and 1 of the vector), and the 16 column groups of a row meet in a 5-shuffle butterfly.
//    FP64: rows 2rg, 2rg+1 and eight columns, an 8-lane reduction of 3 shuffles and 3 adds
//    (GB300's FP64 pipe bounds the FP64 kernel, so adds count).  A quarter-warp's 16-byte
//    loads cover 8 distinct bank groups in both layouts.
//  * FP32 blocks are refined in FP64 against the exact Gram block (sliced-ELL copy):
//    res = u - G_i y, y += L^{-T} L^{-1} res, until ||res|| <= tol ||u|| (refine_tol, or
//    the relaxed inner tolerance of the lane inside CG iterations).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"
#include "proj_ring.cuh"

namespace cimmino {

namespace {

using namespace ring;

// Chain-step row products of a 64 x 64 tile with a vector, 16 FMAs per thread per tile.
// FP32: thread (rg, cg) = (tid / 16, tid % 16) owns rows 4rg..4rg+3 and columns
// 4cg..4cg+3 (4 x 4 register block).
__device__ __forceinline__ void tile_rows(const float *L, const float *v, int rg, int cg,
                                          float (&a)[4]) {
  const float4 x = *reinterpret_cast<const float4 *>(v + 4 * cg);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 l = *reinterpret_cast<const float4 *>(L + (4 * rg + i) * T + 4 * cg);
    a[i] = fma(l.x, x.x, a[i]);
    a[i] = fma(l.y, x.y, a[i]);
    a[i] = fma(l.z, x.z, a[i]);
    a[i] = fma(l.w, x.w, a[i]);
  }
}
// FP64: thread (rg, cg) = (tid / 8, tid % 8) owns rows 2rg, 2rg+1 and the column pairs
// 2cg + 16k, 2cg + 16k + 1 (k < 4): a quarter-warp's 16-byte loads cover one contiguous
// 128-byte row segment (no bank conflict), and the row sums need an 8-lane reduction of
// 3 shuffles and 3 adds instead of 5 and 5 (GB300's FP64 pipe is this kernel's bound).
__device__ __forceinline__ void tile_rows(const double *L, const double *v, int rg, int cg,
                                          double (&a)[2]) {
  double2 x[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) x[k] = *reinterpret_cast<const double2 *>(v + 16 * k + 2 * cg);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double *Lr = L + (2 * rg + i) * T + 2 * cg;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 l = *reinterpret_cast<const double2 *>(Lr + 16 * k);
      a[i] = fma(l.x, x[k].x, a[i]);
      a[i] = fma(l.y, x[k].y, a[i]);
    }
  }
}

// Block-packed triangular tile times v by one warp (FP32 blocks).  Lane p owns row pair
// (p, 63 - p), b = p / 16: the pair's 80 values are 20 16-byte chunks of whole 16-wide
// sub-tile segments, so every chunk multiplies one aligned chunk of v (a broadcast within
// each half-warp).  The chunks split into three fixed ranges: those of the first row,
// those of the second row, and 4 in the middle whose row depends on the half-warp.  Pair
// stride 336 bytes: a quarter-warp's 16-byte loads hit 8 distinct bank groups.
//   lower (inv(L_II)):   row p columns 0 .. 16 (b+1) - 1, row 63 - p columns 0 .. 16 (4-b) - 1
//   upper (inv(L_II)^T): row p columns 16 b .. 63,        row 63 - p columns 16 (3-b) .. 63
__device__ __forceinline__ void dot4(float4 d, float4 x, float &s0, float &s1) {
  s0 = fmaf(d.x, x.x, s0);
  s1 = fmaf(d.y, x.y, s1);
  s0 = fmaf(d.z, x.z, s0);
  s1 = fmaf(d.w, x.w, s1);
}
template <bool UPPER>
__device__ __forceinline__ void bpacked_rows_warp(const float *P, const float *v, float *o,
                                                  int p) {
  const float4 *R = reinterpret_cast<const float4 *>(P + p * kBPackPair);
  const float4 *V = reinterpret_cast<const float4 *>(v);
  const int b = p >> 4;
  float a0 = 0.f, a1 = 0.f, c0 = 0.f, c1 = 0.f;
  if (!UPPER) {
#pragma unroll
    for (int q = 0; q < 4; ++q) dot4(R[q], V[q], a0, a1);
    if (b) {
#pragma unroll
      for (int q = 4; q < 8; ++q) dot4(R[q], V[q], a0, a1);
    } else {
#pragma unroll
      for (int q = 4; q < 8; ++q) dot4(R[q], V[q - 4], c0, c1);
    }
    const int sh = 4 * (b + 1);
#pragma unroll
    for (int q = 8; q < 20; ++q) dot4(R[q], V[q - sh], c0, c1);
  } else {
#pragma unroll
    for (int q = 0; q < 12; ++q) dot4(R[q], V[4 * b + q], a0, a1);
    if (!b) {
#pragma unroll
      for (int q = 12; q < 16; ++q) dot4(R[q], V[q], a0, a1);
    } else {
#pragma unroll
      for (int q = 12; q < 16; ++q) dot4(R[q], V[q - 4], c0, c1);
    }
#pragma unroll
    for (int q = 16; q < 20; ++q) dot4(R[q], V[q - 4], c0, c1);
  }
  o[p] = a0 + a1;
  o[T - 1 - p] = c0 + c1;
}

// Packed triangular tile times v by one warp (FP64 blocks, where every FMA counts on
// GB300's FP64 pipe).  Lane p owns row pair p (rows p and 63 - p,
// kPackPair entries, the second row starting at entry sw): one accumulator runs over the
// pair's entries and is handed over at sw, so every lane does 68 FMAs instead of 128.
//   lower (inv(L_II)):   entry e < sw = p + 1 is (p, e), later (63 - p, e - p - 1)
//   upper (inv(L_II)^T): entry e < sw = 64 - p is (p, p + e), later (63 - p, e - 1)
// Pair stride 544 bytes: a quarter-warp's 16-byte loads hit 4 distinct bank groups.  The
// three padding entries are zero, any in-range index serves.
template <bool UPPER, typename W>
__device__ __forceinline__ void packed_rows_warp(const W *P, const W *v, W *o, int p) {
  constexpr int E = 16 / sizeof(W);
  const W *R = P + p * kPackPair;
  const int sw = UPPER ? 64 - p : p + 1;
  W acc = W(0), first = W(0);
#pragma unroll
  for (int q = 0; q < kPackPair / E; ++q) {
    W d[E];
    if constexpr (E == 4) {
      const float4 x = reinterpret_cast<const float4 *>(R)[q];
      d[0] = x.x;
      d[1] = x.y;
      d[2] = x.z;
      d[3] = x.w;
    } else {
      const double2 x = reinterpret_cast<const double2 *>(R)[q];
      d[0] = x.x;
      d[1] = x.y;
    }
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int e = E * q + j;
      if (e == sw) {
        first = acc;
        acc = W(0);
      }
      int c = UPPER ? (e < sw ? p + e : e - 1) : (e < sw ? e : e - p - 1);
      c = c < T ? c : T - 1;
      acc = fma(d[j], v[c], acc);
    }
  }
  o[p] = first;
  o[T - 1 - p] = acc;
}

// Diagonal-tile products: FP32 blocks stream block-packed triangles of inv(L_II) and
// inv(L_II)^T (2688 of 4096 values, aligned vector reads), FP64 blocks the rectangular full
// packed ones (FP64-bound: 68 instead of 128 FMAs per lane).
template <bool UPPER>
__device__ __forceinline__ void diag_rows(const float *D, const float *v, float *o, int lane) {
  bpacked_rows_warp<UPPER>(D, v, o, lane);
}
template <bool UPPER>
__device__ __forceinline__ void diag_rows(const double *D, const double *v, double *o, int lane) {
  packed_rows_warp<UPPER>(D, v, o, lane);
}

// Sum of a[0..3] over the 16 column groups of a half-warp (5 shuffles, fixed order).
// Returns the sum of row 4rg + row, where row = 2 * lane bit 3 + lane bit 2; all four
// lanes that share those bits hold it.
template <typename W>
__device__ __forceinline__ W reduce_rows(const W (&a)[4], int lane, int &row) {
  const bool hi = (lane & 8) != 0, h2 = (lane & 4) != 0;
  const W s0 = __shfl_xor_sync(0xffffffffu, hi ? a[0] : a[2], 8);
  const W s1 = __shfl_xor_sync(0xffffffffu, hi ? a[1] : a[3], 8);
  const W b0 = (hi ? a[2] : a[0]) + s0;
  const W b1 = (hi ? a[3] : a[1]) + s1;
  const W s2 = __shfl_xor_sync(0xffffffffu, h2 ? b0 : b1, 4);
  W c = (h2 ? b1 : b0) + s2;
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  row = (hi ? 2 : 0) + (h2 ? 1 : 0);
  return c;
}

// FP64 layout: sum of a[0..1] over the 8 column groups of a quarter-warp (3 shuffles,
// fixed order).  Returns the sum of row 2rg + row, row = lane bit 2; the four lanes that
// share that bit hold it.
__device__ __forceinline__ double reduce_rows(const double (&a)[2], int lane, int &row) {
  const bool hi = (lane & 4) != 0;
  const double s = __shfl_xor_sync(0xffffffffu, hi ? a[0] : a[1], 4);
  double c = (hi ? a[1] : a[0]) + s;
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  row = hi ? 1 : 0;
  return c;
}

// Deterministic sum over the 256 consumer threads (fixed order).
__device__ __forceinline__ double csum(double v, double *red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  csync();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < 8; ++w) s += red[w];
  csync();
  return s;
}

// One forward + backward solve: right-hand side in w (overwritten), result in out.
template <typename W>
__device__ void consumer_pass(const Ring &R, const TileRow *__restrict__ tr,
                              const TileRow *__restrict__ trT, int nt, W *w, W *out, uint32_t &t,
                              int32_t *err) {
  const int tid = threadIdx.x, lane = tid & 31;
  constexpr bool D64 = sizeof(W) == 8;
  constexpr int RPT = D64 ? 2 : 4;  // rows per thread in the chain steps
  const int rg = D64 ? tid >> 3 : tid >> 4, cg = D64 ? tid & 7 : tid & 15;
  const bool writer = (lane & 3) == 0;
  int row;
  const int warp = tid >> 5;
  // F0: out_I = inv(L_II) w_I (independent tile rows, one warp per packed tile); every warp
  // still waits for and releases every tile in order, which keeps the slots' phases
  // unambiguous
  for (int I = 0; I < nt; ++I) {
    const W *D = static_cast<const W *>(slot_acquire(R, t, err));
    if ((I & 7) == warp) diag_rows<false>(D, w + I * T, out + I * T, lane);
    slot_release(R, t);
    ++t;
  }
  csync();
  // F1: w_I = out_I - sum_{J<I} N_IJ w_J (sequential over I).  Only the last tile of a
  // row, J = I-1, needs the w of the step just finished, so the barrier that publishes
  // w_{I-1} sits right before that tile and the row's other tiles run while slower warps
  // are still reducing.  A row without that tile ends with the barrier instead, so every
  // w_J is published before any later step reads it.
  for (int I = 0; I < nt; ++I) {
    W a[RPT] = {};
    const int j0 = tr[I].j0;
    for (int J = j0; J < I; ++J) {
      if (J == I - 1) csync();
      tile_rows(static_cast<const W *>(slot_acquire(R, t, err)), w + J * T, rg, cg, a);
      slot_release(R, t);
      ++t;
    }
    const W c = reduce_rows(a, lane, row);
    const int o = I * T + RPT * rg + row;
    if (writer) w[o] = out[o] - c;
    if (j0 >= I) csync();
  }
  csync();
  // B1: w_I = w_I - sum_{J>I} NT_IJ w_J (sequential over I descending); the tiles of a row
  // come in descending J, so the one that needs the previous step, J = I+1, is last
  for (int I = nt - 1; I >= 0; --I) {
    W a[RPT] = {};
    const int j1 = trT[I].j0;
    for (int J = j1; J > I; --J) {
      if (J == I + 1) csync();
      tile_rows(static_cast<const W *>(slot_acquire(R, t, err)), w + J * T, rg, cg, a);
      slot_release(R, t);
      ++t;
    }
    const W c = reduce_rows(a, lane, row);
    if (writer) w[I * T + RPT * rg + row] -= c;
    if (j1 <= I) csync();
  }
  csync();
  // B2: out_I = inv(L_II)^T w_I (packed upper triangles, one warp per tile)
  for (int I = 0; I < nt; ++I) {
    const W *D = static_cast<const W *>(slot_acquire(R, t, err));
    if ((I & 7) == warp) diag_rows<true>(D, w + I * T, out + I * T, lane);
    slot_release(R, t);
    ++t;
  }
  csync();
}

// Producer side of one pass: same tile order as consumer_pass.
__device__ void producer_pass(const Ring &R, const TileRow *__restrict__ tr,
                              const TileRow *__restrict__ trT, int nt, const unsigned char *fac,
                              const unsigned char *dinv, const unsigned char *facT,
                              const unsigned char *dinvT, uint32_t tile_bytes, uint32_t diag_bytes,
                              uint32_t &t, int32_t *err) {
  auto issue = [&](const unsigned char *src) { slot_fill(R, t, src, tile_bytes, err); };
  const size_t TB = tile_bytes;
  const size_t esz = TB / (T * T);
  for (int I = 0; I < nt; ++I) slot_fill(R, t, dinv + (size_t)I * diag_bytes, diag_bytes, err);
  for (int I = 0; I < nt; ++I) {
    const TileRow TI = tr[I];
    const unsigned char *row = fac + (size_t)TI.off * esz;
    for (int J = TI.j0; J < I; ++J) issue(row + (size_t)(J - TI.j0) * TB);
  }
  for (int I = nt - 1; I >= 0; --I) {
    const TileRow U = trT[I];
    const unsigned char *row = facT + (size_t)U.off * esz;
    for (int J = U.j0; J > I; --J) issue(row + (size_t)(J - I - 1) * TB);
  }
  for (int I = 0; I < nt; ++I) slot_fill(R, t, dinvT + (size_t)I * diag_bytes, diag_bytes, err);
}

struct Vecs {
  double *y;  // FP64 solution being refined
  void *w;    // working-precision right-hand side / workspace of a solve pass
  void *out;  // working-precision result of a solve pass
};

// RELAX: inner tolerance of the lane relaxed to min(1e-6, refine_tol / relres_t) (CG
// iterations with refine_relax); otherwise refine_tol.
template <typename W, bool RELAX>
__device__ void consumer_block(const IterArgs &a, const BlockDesc &B, const Ring &R, const Vecs &V,
                               const double *__restrict__ u, double *__restrict__ y, int k,
                               int refine_steps, uint32_t &t, double *red, int *s_again) {
  const int mp = B.nt * T;
  const int tid = threadIdx.x;
  W *w = static_cast<W *>(V.w);
  W *out = static_cast<W *>(V.out);
  const double *ub = u + B.row0 * a.nrhs + k;  // u of this block (stride nrhs), global
  double un2 = 0.0;
  for (int r = tid; r < mp; r += kConsumers) {
    const double ur = r < B.m ? ub[(int64_t)r * a.nrhs] : 0.0;
    V.y[r] = 0.0;
    w[r] = W(ur);
    un2 += ur * ur;
  }
  if (refine_steps > 0)
    un2 = csum(un2, red);  // also orders the writes above
  else
    csync();
  const TileRow *tr = a.trow + B.trow0;
  const TileRow *trT = a.trowT + B.trow0;
  int s = 0;
  for (;;) {
    consumer_pass<W>(R, tr, trT, B.nt, w, out, t, a.err);
    for (int r = tid; r < mp; r += kConsumers) V.y[r] += double(out[r]);
    csync();
    int again = 0;
    if (s < refine_steps) {
      // res = u - G_i y straight into w; a warp covers whole 32-row slices (coalesced) and a
      // thread two rows kConsumers apart at once (two independent load chains in flight;
      // slice widths are uniform across a warp, so the interleaving does not diverge)
      double e2 = 0.0;
      for (int r0 = tid; r0 < mp; r0 += 2 * kConsumers) {
        const int r1 = r0 + kConsumers;
        int wd0 = 0, wd1 = 0;
        const double *sv0 = nullptr, *sv1 = nullptr;
        const int16_t *sc0 = nullptr, *sc1 = nullptr;
        double acc0 = 0.0, acc1 = 0.0;
        if (r0 < B.m) {
          const int sl = B.slice0 + (r0 >> 5), l = r0 & 31;
          const int64_t o = a.soff[sl];
          wd0 = (int)((a.soff[sl + 1] - o) >> 5);
          sv0 = a.sval + o + l;
          sc0 = a.scol + o + l;
          acc0 = ub[(int64_t)r0 * a.nrhs];
        }
        if (r1 < B.m) {
          const int sl = B.slice0 + (r1 >> 5), l = r1 & 31;
          const int64_t o = a.soff[sl];
          wd1 = (int)((a.soff[sl + 1] - o) >> 5);
          sv1 = a.sval + o + l;
          sc1 = a.scol + o + l;
          acc1 = ub[(int64_t)r1 * a.nrhs];
        }
        const int wmax = wd0 > wd1 ? wd0 : wd1;
#pragma unroll 2
        for (int kk = 0; kk < wmax; ++kk) {
          if (kk < wd0) acc0 = fma(-sv0[32 * kk], V.y[sc0[32 * kk]], acc0);
          if (kk < wd1) acc1 = fma(-sv1[32 * kk], V.y[sc1[32 * kk]], acc1);
        }
        if (r0 < mp) w[r0] = W(acc0);  // rows past m (padding) get zero
        if (r1 < mp) w[r1] = W(acc1);
        e2 += acc0 * acc0 + acc1 * acc1;
      }
      e2 = csum(e2, red);
      const double tol = RELAX ? inner_tol(a, 1, (int64_t)B.sys * a.nrhs + k) : a.refine_tol;
      again = e2 > tol * tol * un2;
    }
    if (tid == 0) *s_again = again;
    allsync();
    if (!*(volatile int *)s_again) break;
    ++s;
  }
  for (int r = tid; r < B.m; r += kConsumers) y[(B.row0 + r) * a.nrhs + k] = V.y[r];
  if (tid == 0 && refine_steps > 0) {
    atomicAdd(reinterpret_cast<unsigned long long *>(a.refine_total), (unsigned long long)s);
    atomicMax(a.refine_max, s);
  }
  csync();
}

__device__ void producer_block(const IterArgs &a, const BlockDesc &B, const Ring &R, uint32_t &t,
                               int *s_again) {
  const bool leader = (threadIdx.x & 31) == 0;
  const bool p64 = B.prec64 != 0;
  const unsigned char *fac = p64 ? reinterpret_cast<const unsigned char *>(a.fac64)
                                 : reinterpret_cast<const unsigned char *>(a.fac32);
  const unsigned char *facT = p64 ? reinterpret_cast<const unsigned char *>(a.facT64)
                                  : reinterpret_cast<const unsigned char *>(a.facT32);
  // diagonal tiles: packed triangles (rectangular full packed in FP64, block-packed in FP32)
  const int64_t nd = B.dinv_off / (T * T);  // the block's first diagonal tile
  const unsigned char *dinv = p64 ? reinterpret_cast<const unsigned char *>(a.dinvP64 + nd * kPackTile)
                                  : reinterpret_cast<const unsigned char *>(a.dinvP32 + nd * kBPackTile);
  const unsigned char *dinvT =
      p64 ? reinterpret_cast<const unsigned char *>(a.dinvTP64 + nd * kPackTile)
          : reinterpret_cast<const unsigned char *>(a.dinvTP32 + nd * kBPackTile);
  const uint32_t tb = (uint32_t)(T * T * (p64 ? 8 : 4));
  const uint32_t db = p64 ? (uint32_t)(kPackTile * 8) : (uint32_t)(kBPackTile * 4);
  for (;;) {
    if (leader)
      producer_pass(R, a.trow + B.trow0, a.trowT + B.trow0, B.nt, fac, dinv, facT, dinvT, tb, db,
                    t, a.err);
    __syncwarp();
    allsync();
    if (!*(volatile int *)s_again) break;
  }
}

// ANY64: the context holds FP64 blocks (FP64 precision or fallbacks).  An all-FP32 context
// runs the instance without the FP64 path.  RELAX: CG iterations with refine_relax.  MINB:
// CTAs per SM the registers are budgeted for (1: a deep ring per block; 2: a shallower ring,
// but a second block's chain steps fill the first one's barrier waits); the autotuner picks.
template <bool ANY64, bool RELAX, int MINB>
__global__ void __launch_bounds__(kProjThreads, MINB)
    k_proj(IterArgs a, const double *__restrict__ u, double *__restrict__ y, int check_lane) {
  __shared__ uint64_t full[kMaxProjSlots], empty[kMaxProjSlots];
  __shared__ double red[8];
  __shared__ int s_again, s_abort;
  extern __shared__ __align__(128) unsigned char dsm[];
  const BlockDesc B = a.blk[a.border[blockIdx.x]];  // longest blocks first
  const int mpmax = a.max_mp;
  Ring R;
  R.base = dsm;
  R.full = full;
  R.empty = empty;
  R.slots = (uint32_t)a.proj_slots;
  R.slot_bytes = (uint32_t)a.proj_slot_bytes;
  R.abort = &s_abort;
  Vecs V;
  unsigned char *vb = dsm + (size_t)R.slots * R.slot_bytes;
  const size_t wb = (size_t)a.proj_wbytes * mpmax;
  V.y = reinterpret_cast<double *>(vb);
  V.w = vb + 8 * (size_t)mpmax;
  V.out = vb + 8 * (size_t)mpmax + wb;
  if (threadIdx.x == 0) {
    ring_init(R);
    s_again = 0;
  }
  __syncthreads();
  uint32_t t = 0;  // tiles issued (producer) / consumed (consumers) so far
  const bool producer = threadIdx.x >= kConsumers;
  for (int k = 0; k < a.nrhs; ++k) {
    if (check_lane && a.lane[B.sys * a.nrhs + k].status != CIMMINO_RUNNING) continue;
    const int rs = B.prec64 ? 0 : a.refine_steps;
    if (producer) {
      producer_block(a, B, R, t, &s_again);
    } else if (ANY64 && B.prec64) {
      consumer_block<double, false>(a, B, R, V, u, y, k, 0, t, red, &s_again);
    } else {
      consumer_block<float, RELAX>(a, B, R, V, u, y, k, rs, t, red, &s_again);
    }
  }
  // the producer drains its own copies before the CTA exits (normally already landed)
  if (producer && (threadIdx.x & 31) == 0) ring_drain(R, t);
}

// Watchdog self-test: one thread waits, with the same try_wait loop as the projection
// ring, on an mbarrier that nothing ever completes.  The wait must give up after
// limit_ns and report it in the error word; the spin count is bounded too (2^20 polls), so
// the kernel ends even if the global timer stood still.
__global__ void k_wait_selftest(uint64_t limit_ns, int32_t *err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const uint64_t t0 = global_ns();
  bool done = false;
  for (uint32_t i = 0; i < (1u << 20) && !done; ++i) {
    done = mbar_try_wait(&bar, 0u);
    if (global_ns() - t0 > limit_ns) break;
  }
  if (!done) atomicOr(err, 8);
}

}  // namespace

void launch_wait_selftest(uint64_t limit_ns, int32_t *err, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(limit_ns, err);
}

int proj_smem_bytes(int max_mp, int slots, int slot_bytes, int wbytes) {
  return slots * slot_bytes + 8 * max_mp + 2 * wbytes * max_mp;
}

cudaError_t set_proj_smem_attr(int bytes) {
  const void *fs[8] = {(const void *)k_proj<false, false, 1>, (const void *)k_proj<false, true, 1>,
                       (const void *)k_proj<true, false, 1>,  (const void *)k_proj<true, true, 1>,
                       (const void *)k_proj<false, false, 2>, (const void *)k_proj<false, true, 2>,
                       (const void *)k_proj<true, false, 2>,  (const void *)k_proj<true, true, 2>};
  for (const void *f : fs) {
    const cudaError_t e =
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void launch_proj(const IterArgs &a, const double *u, double *y, int check_lane, cudaStream_t s) {
  if (a.nrhs > 1 && a.proj_rg > 0) {
    launch_proj_mr(a, u, y, check_lane, s);
    return;
  }
  const bool any64 = a.proj_wbytes == 8, relax = a.refine_relax && check_lane;
  auto k = a.proj_minb == 2
               ? (any64 ? (relax ? k_proj<true, true, 2> : k_proj<true, false, 2>)
                        : (relax ? k_proj<false, true, 2> : k_proj<false, false, 2>))
               : (any64 ? (relax ? k_proj<true, true, 1> : k_proj<true, false, 1>)
                        : (relax ? k_proj<false, true, 1> : k_proj<false, false, 1>));
  k<<<a.nblk, kProjThreads, a.proj_smem, s>>>(a, u, y, check_lane);
}

}  // namespace cimmino
