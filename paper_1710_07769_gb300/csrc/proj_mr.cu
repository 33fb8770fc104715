// Multi-right-hand-side projection kernel: Y_i = G_i^{-1} U_i for every block i and a
// group of RG right-hand sides at once (the inner solves of Algorithm 2 step 5 for RG
// independent CG lanes sharing the factors), one CTA per block.  Every factor tile is
// streamed from HBM once per group instead of once per right-hand side.
//
// Same four phases as the single-vector kernel (L = diag(L_II)(I + N)):
//   F0: W_I = inv(L_II) W_I          F1: W_I -= sum_{J<I} N_IJ W_J   (I ascending)
//   B1: W_I -= sum_{J>I} NT_IJ W_J   B2: W_I = inv(L_II)^T W_I       (B1: I descending)
// with W = [row][RG] in shared memory.  Each tile product is a small GEMM
// (64 x 64) . (64 x RG), computed from the TRANSPOSED tile so that a column of the
// operator is a contiguous row in shared memory:
//   F0 streams inv(L_II)^T, F1 streams NT_JI (= N_IJ^T, column I of transposed row J),
//   B1 streams N_JI (= NT_IJ^T), B2 streams inv(L_II).
// Thread layout (8 consumer warps): warp w owns columns k = 8w .. 8w+7 of every tile;
// inside a warp, lane = h + H (g + G s) owns rows MR g .. MR g + MR - 1 and right-hand
// sides NR h .. NR h + NR - 1 and the columns k = 8w + s + S j.  A chain step sums its
// tiles in registers, then reduces over s (shuffles), over the warp pairs (w, w + 4)
// and finally over the four pair sums, always in the same order (deterministic).
//
// FP32 blocks are refined in FP64 against the exact Gram block (sliced-ELL copy), with
// y accumulated in the global output:  res = u - G_i y,  y += L^{-T} L^{-1} res,
// until every active lane has ||res|| <= tol ||u|| (refine_tol, or the lane's relaxed inner
// tolerance inside CG iterations), or the step limit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"
#include "proj_ring.cuh"

namespace cimmino {

namespace {

using namespace ring;

// FP32: 8 x 8 register tiles (shared-memory bound, so large tiles); FP64: small tiles with
// no shuffle reduction (every FP64 add costs as much as an FMA on GB300's FP64 pipe).
template <typename W, int RG>
struct Mr {
  static constexpr int MR = sizeof(W) == 4 ? 8 : (RG == 8 ? 2 : 4);  // rows per lane
  static constexpr int NR = 8;                                         // rhs per lane
  static constexpr int G = T / MR;                                     // row groups
  static constexpr int H = RG / NR;                                    // rhs groups
  static constexpr int S = 32 / (G * H);  // column interleave inside a warp
  static constexpr int KL = 8 / S;        // columns per lane and tile
  static constexpr int E = 16 / sizeof(W);                  // entries per 16-byte vector
  static constexpr int CPL = MR * NR / E;                   // 16-byte chunks per lane tile
  static constexpr int LANE_BYTES = 16 * (CPL + 1);         // padded: conflict-free chunks
  static constexpr int SLOT_BYTES = (32 / S) * LANE_BYTES;  // one warp's partial tile
  static_assert(G * H * S == 32 && KL * S == 8, "lane decomposition");
};

__device__ __forceinline__ float4 vadd(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ double2 vadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ float4 vsub(float4 a, float4 b) {
  return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ double2 vsub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
template <typename W>
struct V16;
template <>
struct V16<float> {
  using type = float4;
  static __device__ __forceinline__ float4 pack(const float *v) {
    return make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct V16<double> {
  using type = double2;
  static __device__ __forceinline__ double2 pack(const double *v) {
    return make_double2(v[0], v[1]);
  }
};

// N consecutive values from 16-byte aligned shared memory
template <int N>
__device__ __forceinline__ void ld16(const float *p, float (&v)[N]) {
#pragma unroll
  for (int q = 0; q < N / 4; ++q) {
    const float4 x = reinterpret_cast<const float4 *>(p)[q];
    v[4 * q] = x.x;
    v[4 * q + 1] = x.y;
    v[4 * q + 2] = x.z;
    v[4 * q + 3] = x.w;
  }
}
template <int N>
__device__ __forceinline__ void ld16(const double *p, double (&v)[N]) {
#pragma unroll
  for (int q = 0; q < N / 2; ++q) {
    const double2 x = reinterpret_cast<const double2 *>(p)[q];
    v[2 * q] = x.x;
    v[2 * q + 1] = x.y;
  }
}

template <typename W, int RG>
struct Lane {
  int g, h, kb;  // row group, right-hand-side group, first column of this lane
  bool lead;     // s == 0: holds the warp's sum after the shuffle reduction
  __device__ Lane() {
    using C = Mr<W, RG>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    h = lane % C::H;
    g = (lane / C::H) % C::G;
    const int s = lane / (C::H * C::G);
    kb = 8 * warp + s;
    lead = s == 0;
  }
};

// acc += At(cols of this lane)^T-part . Wj: At[k * T + r] = A(r, k), Wj[k * RG + c]
template <typename W, int RG>
__device__ __forceinline__ void mr_tile(const W *At, const W *Wj, const Lane<W, RG> &L,
                                        W (&acc)[Mr<W, RG>::MR][Mr<W, RG>::NR]) {
  using C = Mr<W, RG>;
#pragma unroll
  for (int j = 0; j < C::KL; ++j) {
    const int k = L.kb + C::S * j;
    W a[C::MR], b[C::NR];
    ld16<C::MR>(At + k * T + C::MR * L.g, a);
    ld16<C::NR>(Wj + k * RG + C::NR * L.h, b);
#pragma unroll
    for (int i = 0; i < C::MR; ++i)
#pragma unroll
      for (int c = 0; c < C::NR; ++c) acc[i][c] = fma(a[i], b[c], acc[i][c]);
  }
}

template <typename W, int RG>
__device__ __forceinline__ void mr_zero(W (&acc)[Mr<W, RG>::MR][Mr<W, RG>::NR]) {
#pragma unroll
  for (int i = 0; i < Mr<W, RG>::MR; ++i)
#pragma unroll
    for (int c = 0; c < Mr<W, RG>::NR; ++c) acc[i][c] = W(0);
}

// Sum of all lanes' partial tiles: shuffles over s, then warps 4..7 hand their partial
// tiles to warps 0..3 through red, which then holds the four pair sums (w, w + 4).  Each
// lead lane owns a padded region of red (LANE_BYTES), written as 16-byte chunks.
template <typename W, int RG>
__device__ __forceinline__ void mr_reduce(W (&acc)[Mr<W, RG>::MR][Mr<W, RG>::NR],
                                          unsigned char *red, const Lane<W, RG> &L) {
  using C = Mr<W, RG>;
  using VT = typename V16<W>::type;
#pragma unroll
  for (int o = C::G * C::H; o < 32; o <<= 1)
#pragma unroll
    for (int i = 0; i < C::MR; ++i)
#pragma unroll
      for (int c = 0; c < C::NR; ++c) acc[i][c] += __shfl_xor_sync(0xffffffffu, acc[i][c], o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  VT *dst = reinterpret_cast<VT *>(red + (warp & 3) * C::SLOT_BYTES + lane * C::LANE_BYTES);
  const W *flat = &acc[0][0];
  if (warp >= 4 && L.lead) {
#pragma unroll
    for (int q = 0; q < C::CPL; ++q) dst[q] = V16<W>::pack(flat + q * C::E);
  }
  csync();
  if (warp < 4 && L.lead) {
#pragma unroll
    for (int q = 0; q < C::CPL; ++q) dst[q] = vadd(V16<W>::pack(flat + q * C::E), dst[q]);
  }
  csync();
}

// W_I = sum (SUB = false) or W_I -= sum (SUB = true), sum = ((r0 + r1) + r2) + r3.
// Chunk q of lead lane l = h + H g holds rows MR g + i, rhs NR h + c (i NR + c = q E ..).
template <typename W, int RG, bool SUB>
__device__ __forceinline__ void mr_combine(W *WI, const unsigned char *red) {
  using C = Mr<W, RG>;
  using VT = typename V16<W>::type;
  constexpr int NCH = (32 / C::S) * C::CPL;
  for (int ci = threadIdx.x; ci < NCH; ci += kConsumers) {
    const int l = ci / C::CPL, q = ci % C::CPL;
    const unsigned char *src = red + l * C::LANE_BYTES + q * 16;
    const VT s = vadd(vadd(vadd(*reinterpret_cast<const VT *>(src),
                                *reinterpret_cast<const VT *>(src + C::SLOT_BYTES)),
                           *reinterpret_cast<const VT *>(src + 2 * C::SLOT_BYTES)),
                      *reinterpret_cast<const VT *>(src + 3 * C::SLOT_BYTES));
    const int h = l % C::H, g = l / C::H;
    const int idx = q * C::E, i = idx / C::NR, c = idx % C::NR;
    VT *o = reinterpret_cast<VT *>(WI + (C::MR * g + i) * RG + C::NR * h + c);
    *o = SUB ? vsub(*o, s) : s;
  }
  csync();
}

// One forward + backward solve of the RG columns of Wv (overwritten by the result).
template <typename W, int RG>
__device__ void mr_pass(const Ring &R, const TileRow *__restrict__ tr,
                        const TileRow *__restrict__ trT, int nt, W *Wv, unsigned char *red,
                        uint32_t &t,
                        int32_t *err) {
  using C = Mr<W, RG>;
  const Lane<W, RG> L;
  W acc[C::MR][C::NR];
  auto tile = [&](const W *Wj) {
    mr_tile<W, RG>(static_cast<const W *>(slot_acquire(R, t, err)), Wj, L, acc);
    slot_release(R, t);
    ++t;
  };
  constexpr int V = T * RG;  // entries of one tile row of W
  // F0: W_I = inv(L_II) W_I
  for (int I = 0; I < nt; ++I) {
    mr_zero<W, RG>(acc);
    tile(Wv + I * V);
    mr_reduce<W, RG>(acc, red, L);
    mr_combine<W, RG, false>(Wv + I * V, red);
  }
  // F1: W_I -= sum_{J0(I) <= J < I} N_IJ W_J
  for (int I = 0; I < nt; ++I) {
    const int j0 = tr[I].j0;
    if (j0 >= I) continue;
    mr_zero<W, RG>(acc);
    for (int J = j0; J < I; ++J) tile(Wv + J * V);
    mr_reduce<W, RG>(acc, red, L);
    mr_combine<W, RG, true>(Wv + I * V, red);
  }
  // B1: W_I -= sum_{I < J <= J1(I), J0(J) <= I} NT_IJ W_J
  for (int I = nt - 1; I >= 0; --I) {
    const int j1 = trT[I].j0;
    int cnt = 0;
    mr_zero<W, RG>(acc);
    for (int J = I + 1; J <= j1; ++J) {
      if (tr[J].j0 > I) continue;  // zero tile, not streamed
      tile(Wv + J * V);
      ++cnt;
    }
    if (cnt == 0) continue;
    mr_reduce<W, RG>(acc, red, L);
    mr_combine<W, RG, true>(Wv + I * V, red);
  }
  // B2: W_I = inv(L_II)^T W_I
  for (int I = 0; I < nt; ++I) {
    mr_zero<W, RG>(acc);
    tile(Wv + I * V);
    mr_reduce<W, RG>(acc, red, L);
    mr_combine<W, RG, false>(Wv + I * V, red);
  }
}

// Producer side of one pass: the transposed tiles in mr_pass order.
__device__ void mr_producer_pass(const Ring &R, const TileRow *__restrict__ tr,
                                 const TileRow *__restrict__ trT, int nt,
                                 const unsigned char *fac, const unsigned char *dinv,
                                 const unsigned char *facT, const unsigned char *dinvT,
                                 uint32_t tile_bytes, uint32_t &t, int32_t *err) {
  const size_t TB = tile_bytes;
  const size_t esz = TB / (T * T);
  for (int I = 0; I < nt; ++I) slot_fill(R, t, dinvT + (size_t)I * TB, tile_bytes, err);
  for (int I = 0; I < nt; ++I)
    for (int J = tr[I].j0; J < I; ++J)  // NT_JI: column I of transposed tile row J
      slot_fill(R, t, facT + (size_t)trT[J].off * esz + (size_t)(I - J - 1) * TB, tile_bytes,
                err);
  for (int I = nt - 1; I >= 0; --I) {
    const int j1 = trT[I].j0;
    for (int J = I + 1; J <= j1; ++J) {
      const TileRow TJ = tr[J];
      if (TJ.j0 > I) continue;  // N_JI: column I of tile row J
      slot_fill(R, t, fac + (size_t)TJ.off * esz + (size_t)(I - TJ.j0) * TB, tile_bytes, err);
    }
  }
  for (int I = 0; I < nt; ++I) slot_fill(R, t, dinv + (size_t)I * TB, tile_bytes, err);
}

// Per right-hand side g (= thread index mod RG) sum over all 256 consumer threads, fixed
// order; result in out[g].  tmp: 8 * RG doubles.
template <int RG>
__device__ __forceinline__ void rg_sum(double v, double *tmp, double *out) {
#pragma unroll
  for (int o = RG; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < RG) tmp[warp * RG + lane] = v;
  csync();
  if (threadIdx.x < RG) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += tmp[w * RG + threadIdx.x];
    out[threadIdx.x] = s;
  }
  csync();
}

struct Small {
  double *tmp;  // 8 * RG
  double *un2;  // RG: ||u||^2 per right-hand side
  double *e2;   // RG: ||res||^2 per right-hand side
};

template <typename W, int RG>
__device__ void mr_block(const IterArgs &a, const BlockDesc &B, const Ring &R, W *Wv,
                         unsigned char *red,
                         const Small &sm, const double *__restrict__ u, double *__restrict__ y,
                         int k0, uint32_t mask, int refine_steps, int check_lane, uint32_t &t,
                         int *s_again) {
  const int mp = B.nt * T;
  const int tid = threadIdx.x;
  const int64_t ld = a.nrhs;
  // load U (inactive or missing right-hand sides as zeros); thread tid always has g = tid % RG
  double un2 = 0.0;
  for (int e = tid; e < mp * RG; e += kConsumers) {
    const int r = e / RG, g = e % RG;
    double v = 0.0;
    if (r < B.m && ((mask >> g) & 1u)) v = u[(B.row0 + r) * ld + k0 + g];
    Wv[e] = W(v);
    un2 += v * v;
  }
  if (refine_steps > 0)
    rg_sum<RG>(un2, sm.tmp, sm.un2);  // also orders the writes above
  else
    csync();
  const TileRow *tr = a.trow + B.trow0;
  const TileRow *trT = a.trowT + B.trow0;
  int s = 0;
  for (;;) {
    mr_pass<W, RG>(R, tr, trT, B.nt, Wv, red, t, a.err);
    // y (+)= W, in the global output (read back by the refinement residual)
    for (int e = tid; e < B.m * RG; e += kConsumers) {
      const int r = e / RG, g = e % RG;
      if (!((mask >> g) & 1u)) continue;
      double *yp = y + (B.row0 + r) * ld + k0 + g;
      *yp = s == 0 ? double(Wv[e]) : *yp + double(Wv[e]);
    }
    csync();
    int again = 0;
    if (s < refine_steps) {
      // res = u - G_i y into Wv; a warp covers whole 32-row slices of the Gram copy
      double e2[RG];
#pragma unroll
      for (int g = 0; g < RG; ++g) e2[g] = 0.0;
      for (int r = tid; r < mp; r += kConsumers) {
        W *wr = Wv + r * RG;
        if (r >= B.m) {
#pragma unroll
          for (int g = 0; g < RG; ++g) wr[g] = W(0);
          continue;
        }
        double acc[RG];
        const double *ur = u + (B.row0 + r) * ld + k0;
#pragma unroll
        for (int g = 0; g < RG; ++g) acc[g] = ((mask >> g) & 1u) ? ur[g] : 0.0;
        gram_row_residual<RG>(a, B, r, y, ld, k0, mask, acc);
#pragma unroll
        for (int g = 0; g < RG; ++g) {
          wr[g] = W(acc[g]);
          e2[g] += acc[g] * acc[g];
        }
      }
      // per right-hand side totals: warp sums, then the 8 warps in order
      const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
      for (int g = 0; g < RG; ++g) {
        const double v = warp_sum(e2[g]);
        if (lane == 0) sm.tmp[warp * RG + g] = v;
      }
      csync();
      if (tid < RG) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) v += sm.tmp[w * RG + tid];
        sm.e2[tid] = v;
      }
      csync();
      for (int g = 0; g < RG; ++g) {
        if (!((mask >> g) & 1u)) continue;
        const double tol = inner_tol(a, check_lane, (int64_t)B.sys * a.nrhs + k0 + g);
        if (sm.e2[g] > tol * tol * sm.un2[g]) again = 1;
      }
    }
    if (tid == 0) *s_again = again;
    allsync();
    if (!*(volatile int *)s_again) break;
    ++s;
  }
  if (tid == 0 && refine_steps > 0) {
    atomicAdd(reinterpret_cast<unsigned long long *>(a.refine_total),
              (unsigned long long)s * (unsigned long long)__popc(mask));
    atomicMax(a.refine_max, s);
  }
  csync();
}

__device__ void mr_producer_block(const IterArgs &a, const BlockDesc &B, const Ring &R,
                                  uint32_t &t, int *s_again) {
  const bool leader = (threadIdx.x & 31) == 0;
  const bool p64 = B.prec64 != 0;
  const unsigned char *fac = p64 ? reinterpret_cast<const unsigned char *>(a.fac64)
                                 : reinterpret_cast<const unsigned char *>(a.fac32);
  const unsigned char *facT = p64 ? reinterpret_cast<const unsigned char *>(a.facT64)
                                  : reinterpret_cast<const unsigned char *>(a.facT32);
  const unsigned char *dinv = p64 ? reinterpret_cast<const unsigned char *>(a.dinv64 + B.dinv_off)
                                  : reinterpret_cast<const unsigned char *>(a.dinv32 + B.dinv_off);
  const unsigned char *dinvT = p64
                                   ? reinterpret_cast<const unsigned char *>(a.dinvT64 + B.dinv_off)
                                   : reinterpret_cast<const unsigned char *>(a.dinvT32 + B.dinv_off);
  const uint32_t tb = (uint32_t)(T * T * (p64 ? 8 : 4));
  for (;;) {
    if (leader)
      mr_producer_pass(R, a.trow + B.trow0, a.trowT + B.trow0, B.nt, fac, dinv, facT, dinvT, tb,
                       t, a.err);
    __syncwarp();
    allsync();
    if (!*(volatile int *)s_again) break;
  }
}

template <int RG>
__global__ void __launch_bounds__(kProjThreads, 1)
    k_proj_mr(IterArgs a, const double *__restrict__ u, double *__restrict__ y, int check_lane) {
  __shared__ uint64_t full[kMaxProjSlots], empty[kMaxProjSlots];
  __shared__ double tmp[8 * RG], un2[RG], e2[RG];
  __shared__ int s_again, s_abort;
  extern __shared__ __align__(128) unsigned char dsm[];
  // longest blocks first, after the ones the tensor-core kernel takes
  const BlockDesc B = a.blk[a.mr_list[a.mr_ntc + blockIdx.x]];
  Ring R;
  R.base = dsm;
  R.full = full;
  R.empty = empty;
  R.slots = (uint32_t)a.proj_mr_slots;
  R.slot_bytes = (uint32_t)a.proj_slot_bytes;
  R.abort = &s_abort;
  unsigned char *vb = dsm + (size_t)R.slots * R.slot_bytes;
  void *Wv = vb;
  unsigned char *red = vb + (size_t)a.max_mp * RG * a.proj_wbytes;
  const Small sm{tmp, un2, e2};
  if (threadIdx.x == 0) {
    ring_init(R);
    s_again = 0;
  }
  __syncthreads();
  uint32_t t = 0;
  const bool producer = threadIdx.x >= kConsumers;
  for (int k0 = 0; k0 < a.nrhs; k0 += RG) {
    const int ng = min(RG, a.nrhs - k0);
    uint32_t mask = 0;
    for (int g = 0; g < ng; ++g)
      if (!check_lane || a.lane[B.sys * a.nrhs + k0 + g].status == CIMMINO_RUNNING)
        mask |= 1u << g;
    if (!mask) continue;
    if (producer) {
      mr_producer_block(a, B, R, t, &s_again);
    } else if (B.prec64) {
      mr_block<double, RG>(a, B, R, static_cast<double *>(Wv), red, sm, u, y, k0, mask, 0,
                           check_lane, t, &s_again);
    } else {
      mr_block<float, RG>(a, B, R, static_cast<float *>(Wv), red, sm, u, y, k0, mask,
                          a.refine_steps, check_lane, t, &s_again);
    }
  }
  if (producer && (threadIdx.x & 31) == 0) ring_drain(R, t);
}

}  // namespace

int proj_mr_smem_bytes(int max_mp, int rg, int slots, int slot_bytes, int wbytes) {
  int red;
  if (wbytes == 4)
    red = rg == 16 ? Mr<float, 16>::SLOT_BYTES : Mr<float, 8>::SLOT_BYTES;
  else
    red = rg == 16 ? Mr<double, 16>::SLOT_BYTES : Mr<double, 8>::SLOT_BYTES;
  return slots * slot_bytes + max_mp * rg * wbytes + 4 * red;
}

cudaError_t set_proj_mr_smem_attr(int rg, int bytes) {
  if (rg == 16)
    return cudaFuncSetAttribute(k_proj_mr<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return cudaFuncSetAttribute(k_proj_mr<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

void launch_proj_mr(const IterArgs &a, const double *u, double *y, int check_lane,
                    cudaStream_t s) {
  if (a.mr_ntc > 0) launch_proj_mr_tc(a, u, y, check_lane, s);
  const int rest = a.nblk - a.mr_ntc;
  if (rest <= 0) return;
  if (a.proj_rg == 16)
    k_proj_mr<16><<<rest, kProjThreads, a.proj_mr_smem, s>>>(a, u, y, check_lane);
  else
    k_proj_mr<8><<<rest, kProjThreads, a.proj_mr_smem, s>>>(a, u, y, check_lane);
}

}  // namespace cimmino
