// Per-iteration kernels of Algorithm 2 (CG on H x = xi, Section 1.1):
//   k_spmv_res   u = A p (projection input) and the true residual of the current x
//                (||f - A x||_2 through the scaled system: (f - A x)_orig = D (f_s - A_s x))
//   k_proj       y_i = G_i^{-1} u_i per block (proj_kernel.cu)
//   k_spmv_t     psi = A^T y = sum_i A_i^T y_i (gather over the transpose: no atomics)
//                fused with p^T psi
//   k_update_xr  x += alpha p, r -= alpha psi, fused with r^T r
//   k_update_p   p = r + beta p
// Reductions are deterministic: every CTA covers rows of one system only, writes
// its partial sums, and the last CTA to arrive (threadfence + counter) sums the
// partials of its system in a fixed order and updates the per-lane CG state.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace cimmino {

namespace {

constexpr int kThreads = kVecRows;  // one thread per row; CTA table rows per CTA
constexpr int T = kTile;
constexpr int kWarps = kThreads / 32;

// partial-sum kinds
enum { kPartRes = 0, kPartPq = 1, kPartRr = 2, kPartMisc = 3, kNumParts = 4 };

__device__ __forceinline__ double *part_ptr(const IterArgs &a, int kind) {
  return a.part + (int64_t)kind * a.ncta * a.nrhs;
}

// Returns true in the last CTA (of the system's CTAs) to finish.
__device__ __forceinline__ bool arrive_last(int32_t *counter, int ncta) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    int prev = atomicAdd(counter, 1);
    s_last = (prev == ncta - 1);
    if (s_last) *counter = 0;  // reset for the next launch (all CTAs have arrived)
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Sum of the partials of one system for rhs k in a fixed order, by the whole CTA (each
// thread loads a few partials, independent loads in flight, then a fixed tree); every
// thread of the CTA must call it and gets the result.
__device__ __forceinline__ double reduce_partials(const double *part, const SysDesc &S, int nrhs,
                                                  int k, double *red) {
  // four independent accumulators keep four L2 loads in flight per thread; they are
  // combined in a fixed tree, so the result depends only on ncta and the CTA size
  const double *p = part + (int64_t)S.cta0 * nrhs + k;
  const int step = blockDim.x;
  double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
  int c = threadIdx.x;
#pragma unroll 1
  for (; c + 3 * step < S.ncta; c += 4 * step) {
    v0 += __ldcg(p + (int64_t)c * nrhs);
    v1 += __ldcg(p + (int64_t)(c + step) * nrhs);
    v2 += __ldcg(p + (int64_t)(c + 2 * step) * nrhs);
    v3 += __ldcg(p + (int64_t)(c + 3 * step) * nrhs);
  }
#pragma unroll 1
  for (; c < S.ncta; c += step) v0 += __ldcg(p + (int64_t)c * nrhs);
  const double t = (v0 + v1) + (v2 + v3);
  return block_sum(t, red);
}

__device__ __forceinline__ bool lane_running(const IterArgs &a, int sys, int k) {
  return a.lane[sys * a.nrhs + k].status == CIMMINO_RUNNING;
}

// ----------------------------------------------------------------------------
// right-hand side: fs[r][k] = F[k][perm(r)] / d[r]; ||f_k||^2 per lane
__global__ void __launch_bounds__(kThreads)
    k_rhs_scale(IterArgs a, const double *__restrict__ Fin, const int32_t *__restrict__ perm) {
  __shared__ double red[32];
  const CtaDesc C = a.cta[blockIdx.x];
  const SysDesc S = a.sys[C.sys];
  const int64_t r = C.row0 + threadIdx.x;
  const bool act = threadIdx.x < C.rows;
  for (int k = 0; k < a.nrhs; ++k) {
    double f2 = 0.0;
    if (act) {
      double fo = Fin[(int64_t)k * a.N + r];  // original order row r (same system range)
      // a non-finite entry makes the sum NaN (squares of finite entries never do: at worst
      // they overflow to +Inf), so the two failures stay apart after the reduction
      f2 = isfinite(fo) ? fo * fo : __longlong_as_double(0x7ff8000000000000ll);
      a.fs[r * a.nrhs + k] = Fin[(int64_t)k * a.N + perm[r]] / a.d[r];
    }
    double s = block_sum(f2, red);
    if (threadIdx.x == 0) part_ptr(a, kPartMisc)[(int64_t)blockIdx.x * a.nrhs + k] = s;
  }
  if (arrive_last(a.cnt + kPartMisc * a.nsys + C.sys, S.ncta)) {
    for (int k = 0; k < a.nrhs; ++k) {
        double f2 = reduce_partials(part_ptr(a, kPartMisc), S, a.nrhs, k, red);
        if (threadIdx.x == 0) {
          LaneState &L = a.lane[C.sys * a.nrhs + k];
          L.fnorm2 = f2;
          L.t = 0;
          L.iters = 0;
          L.relres = f2 > 0.0 ? 1.0 : 0.0;
          // a NaN or Inf entry is an input error of that lane, not a zero right-hand side;
          // finite entries whose squared norm overflows FP64 (above about 1e154) are beyond
          // the solver's range
          L.status = isnan(f2)   ? CIMMINO_EINVAL
                     : isinf(f2) ? CIMMINO_EUNSUPPORTED
                     : f2 > 0.0  ? CIMMINO_RUNNING
                                 : CIMMINO_CONVERGED;
        }
      }
  }
}

// ----------------------------------------------------------------------------
// u = A v (plain SpMV over the scaled permuted rows), for the projection hooks
__global__ void __launch_bounds__(kThreads)
    k_spmv_plain(IterArgs a, const double *__restrict__ v, double *__restrict__ out) {
  const CtaDesc C = a.cta[blockIdx.x];
  if (threadIdx.x >= C.rows) return;
  const int64_t r = C.row0 + threadIdx.x;
  for (int k = 0; k < a.nrhs; ++k) {
    double s = 0.0;
    for (int64_t q = a.rp[r]; q < a.rp[r + 1]; ++q) s = fma(a.va[q], v[(int64_t)a.ci[q] * a.nrhs + k], s);
    out[r * a.nrhs + k] = s;
  }
}

// u = A p and the residual of x (iteration step 1, convergence decision)
__global__ void __launch_bounds__(kThreads) k_spmv_res(IterArgs a) {
  __shared__ double red[32];
  const CtaDesc C = a.cta[blockIdx.x];
  const SysDesc S = a.sys[C.sys];
  const int64_t r = C.row0 + threadIdx.x;
  const bool act = threadIdx.x < C.rows;
  for (int k = 0; k < a.nrhs; ++k) {
    if (!lane_running(a, C.sys, k)) continue;  // uniform across the CTA
    double e2 = 0.0;
    if (act) {
      // sliced-ELL: a warp's 32 rows read their k-th entries as one coalesced load
      const int sl = C.slice0 + (threadIdx.x >> 5), l = threadIdx.x & 31;
      const int64_t o = a.aoff[sl];
      const int wd = (int)((a.aoff[sl + 1] - o) >> 5);
      const double *av = a.aval + o + l;
      const int32_t *ac = a.acol + o + l;
      double su = 0.0, sx = 0.0;
#pragma unroll 4
      for (int e = 0; e < wd; ++e) {
        const double v = av[32 * e];
        const int64_t c = (int64_t)ac[32 * e] * a.nrhs + k;
        su = fma(v, a.p[c], su);
        sx = fma(v, a.x[c], sx);
      }
      a.u[r * a.nrhs + k] = su;
      double e = a.d[r] * (a.fs[r * a.nrhs + k] - sx);
      e2 = e * e;
    }
    double s = block_sum(e2, red);
    if (threadIdx.x == 0) part_ptr(a, kPartRes)[(int64_t)blockIdx.x * a.nrhs + k] = s;
  }
  if (arrive_last(a.cnt + kPartRes * a.nsys + C.sys, S.ncta)) {
    for (int k = 0; k < a.nrhs; ++k) {
        LaneState &L = a.lane[C.sys * a.nrhs + k];
        if (L.status != CIMMINO_RUNNING) continue;  // uniform: read before any update
        double e2 = reduce_partials(part_ptr(a, kPartRes), S, a.nrhs, k, red);
        if (threadIdx.x == 0) {
          double rel = sqrt(e2 / L.fnorm2);
          L.relres = rel;
          if (rel <= a.tol) {
            L.status = CIMMINO_CONVERGED;
            L.iters = L.t;
          } else if (L.t >= a.max_iter) {
            L.status = CIMMINO_ENOCONV;
            L.iters = L.t;
          }
        }
      }
  }
}

// ----------------------------------------------------------------------------
// psi = A^T y (column gather over the transpose); MODE 1 also reduces p^T psi -> alpha
template <int MODE>
__global__ void __launch_bounds__(kThreads)
    k_spmv_t(IterArgs a, const double *__restrict__ yin, double *__restrict__ out) {
  __shared__ double red[32];
  const CtaDesc C = a.cta[blockIdx.x];
  const SysDesc S = a.sys[C.sys];
  const bool act = threadIdx.x < C.rows;
  // column of A (row of the transpose) at this thread's sliced-ELL position
  const int64_t j = act ? (int64_t)a.tord[C.row0 + threadIdx.x] : C.row0 + threadIdx.x;
  for (int k = 0; k < a.nrhs; ++k) {
    if (MODE == 1 && !lane_running(a, C.sys, k)) continue;
    double pq = 0.0;
    if (act) {
      const int sl = C.slice0 + (threadIdx.x >> 5), l = threadIdx.x & 31;
      const int64_t o = a.toff[sl];
      const int wd = (int)((a.toff[sl + 1] - o) >> 5);
      const double *tv = a.tval + o + l;
      const int32_t *tc = a.tcol + o + l;
      double s = 0.0;
#pragma unroll 4
      for (int e = 0; e < wd; ++e) s = fma(tv[32 * e], yin[(int64_t)tc[32 * e] * a.nrhs + k], s);
      out[j * a.nrhs + k] = s;
      if (MODE == 1) pq = a.p[j * a.nrhs + k] * s;
    }
    if (MODE == 1) {
      double t = block_sum(pq, red);
      if (threadIdx.x == 0) part_ptr(a, kPartPq)[(int64_t)blockIdx.x * a.nrhs + k] = t;
    }
  }
  if (MODE == 1 && arrive_last(a.cnt + kPartPq * a.nsys + C.sys, S.ncta)) {
    for (int k = 0; k < a.nrhs; ++k) {
        LaneState &L = a.lane[C.sys * a.nrhs + k];
        if (L.status != CIMMINO_RUNNING) continue;  // uniform: read before any update
        double pq = reduce_partials(part_ptr(a, kPartPq), S, a.nrhs, k, red);
        if (threadIdx.x == 0) {
          L.pq = pq;
          if (!(pq > 0.0) || !isfinite(pq)) {
            L.status = CIMMINO_EBREAKDOWN;
            L.iters = L.t;
            L.alpha = 0.0;
          } else {
            L.alpha = L.rho[L.t & 1] / pq;
          }
        }
      }
  }
}

// r = p = xi, x = 0, rho_0 = r^T r
__global__ void __launch_bounds__(kThreads) k_cg_init(IterArgs a) {
  __shared__ double red[32];
  const CtaDesc C = a.cta[blockIdx.x];
  const SysDesc S = a.sys[C.sys];
  const int64_t j = C.row0 + threadIdx.x;
  const bool act = threadIdx.x < C.rows;
  for (int k = 0; k < a.nrhs; ++k) {
    double rr = 0.0;
    if (act) {
      const int64_t o = j * a.nrhs + k;
      const double v = a.psi[o];
      a.r[o] = v;
      a.p[o] = v;
      a.x[o] = 0.0;
      rr = v * v;
    }
    double t = block_sum(rr, red);
    if (threadIdx.x == 0) part_ptr(a, kPartRr)[(int64_t)blockIdx.x * a.nrhs + k] = t;
  }
  if (arrive_last(a.cnt + kPartRr * a.nsys + C.sys, S.ncta)) {
    for (int k = 0; k < a.nrhs; ++k) {
        double rr = reduce_partials(part_ptr(a, kPartRr), S, a.nrhs, k, red);
        if (threadIdx.x == 0) {
          LaneState &L = a.lane[C.sys * a.nrhs + k];
          L.rho[0] = rr;
          L.rho[1] = rr;
        }
      }
  }
}

// x += alpha p, r -= alpha psi, rho_{t+1} = r^T r, beta
__global__ void __launch_bounds__(kThreads) k_update_xr(IterArgs a) {
  __shared__ double red[32];
  const CtaDesc C = a.cta[blockIdx.x];
  const SysDesc S = a.sys[C.sys];
  const int64_t j = C.row0 + threadIdx.x;
  const bool act = threadIdx.x < C.rows;
  for (int k = 0; k < a.nrhs; ++k) {
    const LaneState &L = a.lane[C.sys * a.nrhs + k];
    if (L.status != CIMMINO_RUNNING) continue;
    const double alpha = L.alpha;
    double rr = 0.0;
    if (act) {
      const int64_t o = j * a.nrhs + k;
      a.x[o] = fma(alpha, a.p[o], a.x[o]);
      const double rn = fma(-alpha, a.psi[o], a.r[o]);
      a.r[o] = rn;
      rr = rn * rn;
    }
    double t = block_sum(rr, red);
    if (threadIdx.x == 0) part_ptr(a, kPartRr)[(int64_t)blockIdx.x * a.nrhs + k] = t;
  }
  if (arrive_last(a.cnt + kPartRr * a.nsys + C.sys, S.ncta)) {
    for (int k = 0; k < a.nrhs; ++k) {
        LaneState &L = a.lane[C.sys * a.nrhs + k];
        if (L.status != CIMMINO_RUNNING) continue;  // uniform: read before any update
        double rr = reduce_partials(part_ptr(a, kPartRr), S, a.nrhs, k, red);
        if (threadIdx.x == 0) {
          const int par = L.t & 1;
          L.rho[par ^ 1] = rr;
          L.beta = rr / L.rho[par];
        }
      }
  }
}

// ----------------------------------------------------------------------------
// The same four per-iteration vector steps for several right-hand sides (CG lanes):
// right-hand sides in chunks of up to KC per row, so every entry of A (or A^T) is read
// once per chunk instead of once per right-hand side, and a row's values [r][k0 .. k0+KC)
// are contiguous; one block reduction covers a whole chunk.
constexpr int KC = 8;

// Sum over the CTA of v[0..kc) (fixed order: warp butterflies, then the warps in order),
// written to part[base + kk].  red: at least KC * kWarps doubles.
__device__ __forceinline__ void chunk_partials(double (&v)[KC], int kc, double *red, double *part,
                                               int64_t base) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int kk = 0; kk < KC; ++kk) v[kk] = warp_sum(v[kk]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) red[kk * kWarps + warp] = v[kk];
  }
  __syncthreads();
  if (threadIdx.x < (unsigned)kc) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += red[threadIdx.x * kWarps + w];
    part[base + threadIdx.x] = t;
  }
}

// u = A p for all lanes and the residual of x (convergence decision of running lanes)
__global__ void __launch_bounds__(kThreads) k_spmv_res_mr(IterArgs a) {
  __shared__ double red[KC * kWarps];
  const CtaDesc C = a.cta[blockIdx.x];
  const SysDesc S = a.sys[C.sys];
  const int64_t r = C.row0 + threadIdx.x;
  const bool act = threadIdx.x < C.rows;
  const int sl = C.slice0 + (threadIdx.x >> 5), l = threadIdx.x & 31;
  const int64_t o = a.aoff[sl];
  const int wd = (int)((a.aoff[sl + 1] - o) >> 5);
  for (int k0 = 0; k0 < a.nrhs; k0 += KC) {
    const int kc = min(KC, a.nrhs - k0);
    double e2[KC];
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) e2[kk] = 0.0;
    if (act) {
      double su[KC], sx[KC];
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) su[kk] = sx[kk] = 0.0;
      if (kc == KC && (a.nrhs & 1) == 0) {  // full chunk, 16-byte aligned: vector loads
        for (int e = 0; e < wd; ++e) {
          const double v = a.aval[o + 32 * e + l];
          const int64_t c = (int64_t)a.acol[o + 32 * e + l] * a.nrhs + k0;
          const double2 *pp = reinterpret_cast<const double2 *>(a.p + c);
          const double2 *xx = reinterpret_cast<const double2 *>(a.x + c);
#pragma unroll
          for (int h = 0; h < KC / 2; ++h) {
            const double2 pv = pp[h], xv = xx[h];
            su[2 * h] = fma(v, pv.x, su[2 * h]);
            su[2 * h + 1] = fma(v, pv.y, su[2 * h + 1]);
            sx[2 * h] = fma(v, xv.x, sx[2 * h]);
            sx[2 * h + 1] = fma(v, xv.y, sx[2 * h + 1]);
          }
        }
      } else {
        for (int e = 0; e < wd; ++e) {
          const double v = a.aval[o + 32 * e + l];
          const int64_t c = (int64_t)a.acol[o + 32 * e + l] * a.nrhs + k0;
#pragma unroll
          for (int kk = 0; kk < KC; ++kk)
            if (kk < kc) {
              su[kk] = fma(v, a.p[c + kk], su[kk]);
              sx[kk] = fma(v, a.x[c + kk], sx[kk]);
            }
        }
      }
#pragma unroll
      for (int kk = 0; kk < KC; ++kk)
        if (kk < kc) {
          const int64_t q = r * a.nrhs + k0 + kk;
          a.u[q] = su[kk];
          const double ev = a.d[r] * (a.fs[q] - sx[kk]);
          e2[kk] = ev * ev;
        }
    }
    chunk_partials(e2, kc, red, part_ptr(a, kPartRes), (int64_t)blockIdx.x * a.nrhs + k0);
  }
  if (arrive_last(a.cnt + kPartRes * a.nsys + C.sys, S.ncta)) {
    for (int k = 0; k < a.nrhs; ++k) {
      LaneState &L = a.lane[C.sys * a.nrhs + k];
      if (L.status != CIMMINO_RUNNING) continue;  // uniform: read before any update
      double e2 = reduce_partials(part_ptr(a, kPartRes), S, a.nrhs, k, red);
      if (threadIdx.x == 0) {
        double rel = sqrt(e2 / L.fnorm2);
        L.relres = rel;
        if (rel <= a.tol) {
          L.status = CIMMINO_CONVERGED;
          L.iters = L.t;
        } else if (L.t >= a.max_iter) {
          L.status = CIMMINO_ENOCONV;
          L.iters = L.t;
        }
      }
    }
  }
}

// psi = A^T y for all lanes, p^T psi -> alpha of running lanes
__global__ void __launch_bounds__(kThreads) k_spmv_t_mr(IterArgs a) {
  __shared__ double red[KC * kWarps];
  const CtaDesc C = a.cta[blockIdx.x];
  const SysDesc S = a.sys[C.sys];
  const bool act = threadIdx.x < C.rows;
  // column of A (row of the transpose) at this thread's sliced-ELL position
  const int64_t j = act ? (int64_t)a.tord[C.row0 + threadIdx.x] : C.row0 + threadIdx.x;
  const int sl = C.slice0 + (threadIdx.x >> 5), l = threadIdx.x & 31;
  const int64_t o = a.toff[sl];
  const int wd = (int)((a.toff[sl + 1] - o) >> 5);
  for (int k0 = 0; k0 < a.nrhs; k0 += KC) {
    const int kc = min(KC, a.nrhs - k0);
    double pq[KC];
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) pq[kk] = 0.0;
    if (act) {
      double sv[KC];
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) sv[kk] = 0.0;
      if (kc == KC && (a.nrhs & 1) == 0) {  // full chunk, 16-byte aligned: vector loads
        for (int e = 0; e < wd; ++e) {
          const double v = a.tval[o + 32 * e + l];
          const int64_t c = (int64_t)a.tcol[o + 32 * e + l] * a.nrhs + k0;
          const double2 *yy = reinterpret_cast<const double2 *>(a.y + c);
#pragma unroll
          for (int h = 0; h < KC / 2; ++h) {
            const double2 yv = yy[h];
            sv[2 * h] = fma(v, yv.x, sv[2 * h]);
            sv[2 * h + 1] = fma(v, yv.y, sv[2 * h + 1]);
          }
        }
      } else {
        for (int e = 0; e < wd; ++e) {
          const double v = a.tval[o + 32 * e + l];
          const int64_t c = (int64_t)a.tcol[o + 32 * e + l] * a.nrhs + k0;
#pragma unroll
          for (int kk = 0; kk < KC; ++kk)
            if (kk < kc) sv[kk] = fma(v, a.y[c + kk], sv[kk]);
        }
      }
#pragma unroll
      for (int kk = 0; kk < KC; ++kk)
        if (kk < kc) {
          const int64_t q = j * a.nrhs + k0 + kk;
          a.psi[q] = sv[kk];
          pq[kk] = a.p[q] * sv[kk];
        }
    }
    chunk_partials(pq, kc, red, part_ptr(a, kPartPq), (int64_t)blockIdx.x * a.nrhs + k0);
  }
  if (arrive_last(a.cnt + kPartPq * a.nsys + C.sys, S.ncta)) {
    for (int k = 0; k < a.nrhs; ++k) {
      LaneState &L = a.lane[C.sys * a.nrhs + k];
      if (L.status != CIMMINO_RUNNING) continue;  // uniform: read before any update
      double pq = reduce_partials(part_ptr(a, kPartPq), S, a.nrhs, k, red);
      if (threadIdx.x == 0) {
        L.pq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) {
          L.status = CIMMINO_EBREAKDOWN;
          L.iters = L.t;
          L.alpha = 0.0;
        } else {
          L.alpha = L.rho[L.t & 1] / pq;
        }
      }
    }
  }
}

// x += alpha p, r -= alpha psi (running lanes), rho_{t+1} = r^T r, beta
__global__ void __launch_bounds__(kThreads) k_update_xr_mr(IterArgs a) {
  __shared__ double red[KC * kWarps];
  const CtaDesc C = a.cta[blockIdx.x];
  const SysDesc S = a.sys[C.sys];
  const int64_t j = C.row0 + threadIdx.x;
  const bool act = threadIdx.x < C.rows;
  const LaneState *LS = a.lane + (int64_t)C.sys * a.nrhs;
  for (int k0 = 0; k0 < a.nrhs; k0 += KC) {
    const int kc = min(KC, a.nrhs - k0);
    double rr[KC];
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) rr[kk] = 0.0;
    if (act) {
#pragma unroll
      for (int kk = 0; kk < KC; ++kk)
        if (kk < kc && LS[k0 + kk].status == CIMMINO_RUNNING) {
          const double alpha = LS[k0 + kk].alpha;
          const int64_t q = j * a.nrhs + k0 + kk;
          a.x[q] = fma(alpha, a.p[q], a.x[q]);
          const double rn = fma(-alpha, a.psi[q], a.r[q]);
          a.r[q] = rn;
          rr[kk] = rn * rn;
        }
    }
    chunk_partials(rr, kc, red, part_ptr(a, kPartRr), (int64_t)blockIdx.x * a.nrhs + k0);
  }
  if (arrive_last(a.cnt + kPartRr * a.nsys + C.sys, S.ncta)) {
    for (int k = 0; k < a.nrhs; ++k) {
      LaneState &L = a.lane[C.sys * a.nrhs + k];
      if (L.status != CIMMINO_RUNNING) continue;  // uniform: read before any update
      double rr = reduce_partials(part_ptr(a, kPartRr), S, a.nrhs, k, red);
      if (threadIdx.x == 0) {
        const int par = L.t & 1;
        L.rho[par ^ 1] = rr;
        L.beta = rr / L.rho[par];
      }
    }
  }
}

// p = r + beta p for running lanes, then t += 1
__global__ void __launch_bounds__(kThreads) k_update_p_mr(IterArgs a) {
  const CtaDesc C = a.cta[blockIdx.x];
  const SysDesc S = a.sys[C.sys];
  const int64_t j = C.row0 + threadIdx.x;
  const LaneState *LS = a.lane + (int64_t)C.sys * a.nrhs;
  if (threadIdx.x < C.rows)
    for (int k = 0; k < a.nrhs; ++k)
      if (LS[k].status == CIMMINO_RUNNING) {
        const int64_t q = j * a.nrhs + k;
        a.p[q] = fma(LS[k].beta, a.p[q], a.r[q]);
      }
  if (blockIdx.x == (unsigned)S.cta0) {
    __syncthreads();
    for (int k = threadIdx.x; k < a.nrhs; k += kThreads) {
      LaneState &L = a.lane[C.sys * a.nrhs + k];
      if (L.status == CIMMINO_RUNNING) L.t += 1;
    }
  }
}

// Flattened element-wise updates for nrhs dividing 32: consecutive threads touch
// consecutive (row, lane) entries of the [row][nrhs] vectors (coalesced), and a thread
// always meets the same lane k = threadIdx.x mod nrhs, so r^T r per lane is a fixed
// shuffle tree over the lanes of a warp with equal k, then the warps in order.
__global__ void __launch_bounds__(kThreads) k_update_xr_fl(IterArgs a) {
  __shared__ double red[kWarps * 32];
  const CtaDesc C = a.cta[blockIdx.x];
  const SysDesc S = a.sys[C.sys];
  const int nr = a.nrhs, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = threadIdx.x % nr;
  const LaneState &Lk = a.lane[C.sys * nr + k];
  const bool run = Lk.status == CIMMINO_RUNNING;
  const double alpha = Lk.alpha;
  double rr = 0.0;
  const int64_t base = C.row0 * nr, cnt = (int64_t)C.rows * nr;
  if (run)
    for (int64_t e = threadIdx.x; e < cnt; e += kThreads) {
      const int64_t q = base + e;
      a.x[q] = fma(alpha, a.p[q], a.x[q]);
      const double rn = fma(-alpha, a.psi[q], a.r[q]);
      a.r[q] = rn;
      rr += rn * rn;
    }
  for (int o = nr; o < 32; o <<= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
  if (lane < nr) red[warp * 32 + lane] = rr;
  __syncthreads();
  if (threadIdx.x < (unsigned)nr) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += red[w * 32 + threadIdx.x];
    part_ptr(a, kPartRr)[(int64_t)blockIdx.x * nr + threadIdx.x] = t;
  }
  if (arrive_last(a.cnt + kPartRr * a.nsys + C.sys, S.ncta)) {
    for (int kk = 0; kk < nr; ++kk) {
      LaneState &L = a.lane[C.sys * nr + kk];
      if (L.status != CIMMINO_RUNNING) continue;  // uniform: read before any update
      double rs = reduce_partials(part_ptr(a, kPartRr), S, nr, kk, red);
      if (threadIdx.x == 0) {
        const int par = L.t & 1;
        L.rho[par ^ 1] = rs;
        L.beta = rs / L.rho[par];
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_update_p_fl(IterArgs a) {
  const CtaDesc C = a.cta[blockIdx.x];
  const SysDesc S = a.sys[C.sys];
  const int nr = a.nrhs;
  const int k = threadIdx.x % nr;
  const LaneState &Lk = a.lane[C.sys * nr + k];
  if (Lk.status == CIMMINO_RUNNING) {
    const double beta = Lk.beta;
    const int64_t base = C.row0 * nr, cnt = (int64_t)C.rows * nr;
    for (int64_t e = threadIdx.x; e < cnt; e += kThreads) {
      const int64_t q = base + e;
      a.p[q] = fma(beta, a.p[q], a.r[q]);
    }
  }
  if (blockIdx.x == (unsigned)S.cta0) {
    __syncthreads();
    if (threadIdx.x < (unsigned)nr) {
      LaneState &L = a.lane[C.sys * nr + threadIdx.x];
      if (L.status == CIMMINO_RUNNING) L.t += 1;
    }
  }
}

// ----------------------------------------------------------------------------
// Algorithm 1 (block Cimmino with relaxation parameter omega, Section 1.1):
//   x <- x + omega * sum_i A_i^+ (f_i - A_i x)
// u = f_s - A x over the scaled permuted rows (the per-block residuals f_i - A_i x)
__global__ void __launch_bounds__(kThreads) k_cim_residual(IterArgs a) {
  const CtaDesc C = a.cta[blockIdx.x];
  if (threadIdx.x >= C.rows) return;
  const int64_t r = C.row0 + threadIdx.x;
  const int sl = C.slice0 + (threadIdx.x >> 5), l = threadIdx.x & 31;
  const int64_t o = a.aoff[sl];
  const int wd = (int)((a.aoff[sl + 1] - o) >> 5);
  for (int k = 0; k < a.nrhs; ++k) {
    double sx = 0.0;
    for (int e = 0; e < wd; ++e)
      sx = fma(a.aval[o + 32 * e + l], a.x[(int64_t)a.acol[o + 32 * e + l] * a.nrhs + k], sx);
    a.u[r * a.nrhs + k] = a.fs[r * a.nrhs + k] - sx;
  }
}

// x += omega psi (psi = sum_i A_i^T y_i, the sum of the block projections)
__global__ void __launch_bounds__(kThreads) k_cim_update(IterArgs a, double omega) {
  const CtaDesc C = a.cta[blockIdx.x];
  if (threadIdx.x >= C.rows) return;
  const int64_t j = C.row0 + threadIdx.x;
  for (int k = 0; k < a.nrhs; ++k) {
    const int64_t o = j * a.nrhs + k;
    a.x[o] = fma(omega, a.psi[o], a.x[o]);
  }
}

// p = r + beta p, then t += 1
__global__ void __launch_bounds__(kThreads) k_update_p(IterArgs a) {
  const CtaDesc C = a.cta[blockIdx.x];
  const SysDesc S = a.sys[C.sys];
  const int64_t j = C.row0 + threadIdx.x;
  for (int k = 0; k < a.nrhs; ++k) {
    const LaneState &L = a.lane[C.sys * a.nrhs + k];
    if (L.status != CIMMINO_RUNNING) continue;
    if (threadIdx.x < C.rows) {
      const int64_t o = j * a.nrhs + k;
      a.p[o] = fma(L.beta, a.p[o], a.r[o]);
    }
  }
  // one CTA per system advances the iteration counters of its running lanes
  if (blockIdx.x == (unsigned)S.cta0) {
    __syncthreads();
    if (threadIdx.x < (unsigned)a.nrhs) {
      LaneState &L = a.lane[C.sys * a.nrhs + threadIdx.x];
      if (L.status == CIMMINO_RUNNING) L.t += 1;
    }
  }
}

// final statistics: per CTA partial max |D(f_s - A_s x)|, sum |x|, max |f|, max row abs-sum
__global__ void __launch_bounds__(kThreads)
    k_final_stats(IterArgs a, const double *__restrict__ Fin, const double *__restrict__ rowabs,
                  double *__restrict__ out) {
  __shared__ double sred[3][kWarps];
  const CtaDesc C = a.cta[blockIdx.x];
  const int64_t r = C.row0 + threadIdx.x;
  const bool act = threadIdx.x < C.rows;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < a.nrhs; ++k) {
    double rmax = 0.0, x1 = 0.0, fmax_ = 0.0;
    if (act) {
      double sx = 0.0;
      for (int64_t q = a.rp[r]; q < a.rp[r + 1]; ++q) sx = fma(a.va[q], a.x[(int64_t)a.ci[q] * a.nrhs + k], sx);
      rmax = fabs(a.d[r] * (a.fs[r * a.nrhs + k] - sx));
      x1 = a.cs ? fabs(a.x[r * a.nrhs + k] / a.cs[r]) : fabs(a.x[r * a.nrhs + k]);
      fmax_ = fabs(Fin[(int64_t)k * a.N + r]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
      x1 += __shfl_xor_sync(0xffffffffu, x1, o);
      fmax_ = fmax(fmax_, __shfl_xor_sync(0xffffffffu, fmax_, o));
    }
    if (lane == 0) {
      sred[0][warp] = rmax;
      sred[1][warp] = x1;
      sred[2][warp] = fmax_;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double m0 = 0, s1 = 0, m2 = 0;
      for (int q = 0; q < kWarps; ++q) {
        m0 = fmax(m0, sred[0][q]);
        s1 += sred[1][q];
        m2 = fmax(m2, sred[2][q]);
      }
      double *o = out + ((int64_t)blockIdx.x * a.nrhs + k) * 4;
      o[0] = m0;
      o[1] = s1;
      o[2] = m2;
      double am = 0.0;
      for (int q = 0; q < C.rows; ++q) am = fmax(am, rowabs[C.row0 + q]);
      o[3] = am;
    }
    __syncthreads();
  }
}

// ||row r of the original A||_1 = d_r * sum_j |S_rj| cs_j (S the scaled permuted matrix)
__global__ void k_row_abs(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ va, const double *__restrict__ d,
                          const double *__restrict__ cs, int64_t N, double *__restrict__ rowabs) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  double s = 0.0;
  if (cs)
    for (int64_t q = rp[r]; q < rp[r + 1]; ++q) s += fabs(va[q]) * cs[ci[q]];
  else
    for (int64_t q = rp[r]; q < rp[r + 1]; ++q) s += fabs(va[q]);
  rowabs[r] = s * d[r];
}

__global__ void k_unscale_cols(double *__restrict__ x, const double *__restrict__ cs, int64_t N,
                               int32_t nrhs) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * nrhs) return;
  x[i] = x[i] / cs[i / nrhs];
}

}  // namespace

// ============================================================================ launchers
void launch_rhs_scale(const IterArgs &a, const double *Fin, const int32_t *perm, cudaStream_t s) {
  k_rhs_scale<<<a.ncta, kThreads, 0, s>>>(a, Fin, perm);
}

void launch_spmv_plain(const IterArgs &a, const double *v, double *out, cudaStream_t s) {
  k_spmv_plain<<<a.ncta, kThreads, 0, s>>>(a, v, out);
}

void launch_spmv_t(const IterArgs &a, const double *y, double *out, cudaStream_t s) {
  k_spmv_t<0><<<a.ncta, kThreads, 0, s>>>(a, y, out);
}

void launch_cg_init(const IterArgs &a, cudaStream_t s) {
  k_cg_init<<<a.ncta, kThreads, 0, s>>>(a);
}

void launch_iteration(const IterArgs &a, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  if (a.nrhs > 1) {
    k_spmv_res_mr<<<a.ncta, kThreads, 0, s>>>(a);
    if (e0) cudaEventRecord(e0, s);
    launch_proj(a, a.u, a.y, 1, s);
    if (e1) cudaEventRecord(e1, s);
    k_spmv_t_mr<<<a.ncta, kThreads, 0, s>>>(a);
    if (32 % a.nrhs == 0) {
      k_update_xr_fl<<<a.ncta, kThreads, 0, s>>>(a);
      k_update_p_fl<<<a.ncta, kThreads, 0, s>>>(a);
    } else {
      k_update_xr_mr<<<a.ncta, kThreads, 0, s>>>(a);
      k_update_p_mr<<<a.ncta, kThreads, 0, s>>>(a);
    }
    return;
  }
  k_spmv_res<<<a.ncta, kThreads, 0, s>>>(a);
  if (e0) cudaEventRecord(e0, s);
  launch_proj(a, a.u, a.y, 1, s);
  if (e1) cudaEventRecord(e1, s);
  k_spmv_t<1><<<a.ncta, kThreads, 0, s>>>(a, a.y, a.psi);
  k_update_xr<<<a.ncta, kThreads, 0, s>>>(a);
  k_update_p<<<a.ncta, kThreads, 0, s>>>(a);
}

void launch_cim_sweep(const IterArgs &a, double omega, cudaStream_t s) {
  k_cim_residual<<<a.ncta, kThreads, 0, s>>>(a);
  launch_proj(a, a.u, a.y, 0, s);
  k_spmv_t<0><<<a.ncta, kThreads, 0, s>>>(a, a.y, a.psi);
  k_cim_update<<<a.ncta, kThreads, 0, s>>>(a, omega);
}

void launch_final_stats(const IterArgs &a, const double *Fin, const double *rowabs, double *out,
                        cudaStream_t s) {
  k_final_stats<<<a.ncta, kThreads, 0, s>>>(a, Fin, rowabs, out);
}

void launch_row_abs(const int64_t *rp, const int32_t *ci, const double *va, const double *d,
                    const double *cs, int64_t N, double *rowabs, cudaStream_t s) {
  k_row_abs<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(rp, ci, va, d, cs, N, rowabs);
}

void launch_unscale_cols(double *x, const double *cs, int64_t N, int32_t nrhs, cudaStream_t s) {
  const int64_t tot = N * nrhs;
  k_unscale_cols<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(x, cs, N, nrhs);
}


// ----------------------------------------------------------------------------
// FP64 FMA throughput probe: every thread runs 8 independent FMA chains; the result is
// written only if it is NaN (never, for the given inputs), so the work cannot be dropped.
namespace {
__global__ void __launch_bounds__(256) k_dfma_probe(int iters, double a, double b, double *sink) {
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s != s) sink[0] = s;
}
}  // namespace

double launch_dfma_probe(int iters, double *sink, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                         int64_t *fmas) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8;  // 8 CTAs x 256 threads per SM
  k_dfma_probe<<<blocks, 256, 0, s>>>(iters / 8, 0.999999, 1e-9, sink);  // warm-up
  cudaEventRecord(e0, s);
  k_dfma_probe<<<blocks, 256, 0, s>>>(iters, 0.999999, 1e-9, sink);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  *fmas = (int64_t)blocks * 256 * 8 * iters;
  return ms;
}
}  // namespace cimmino
