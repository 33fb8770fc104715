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
  double v = 0.0;
  for (int c = threadIdx.x; c < S.ncta; c += blockDim.x)
    v += __ldcg(part + (int64_t)(S.cta0 + c) * nrhs + k);
  return block_sum(v, red);
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
      f2 = fo * fo;
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
          L.status = f2 > 0.0 ? CIMMINO_RUNNING : CIMMINO_CONVERGED;
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
  const int64_t j = C.row0 + threadIdx.x;  // column index (square systems)
  const bool act = threadIdx.x < C.rows;
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
      x1 = fabs(a.x[r * a.nrhs + k]);
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

__global__ void k_row_abs(const int64_t *__restrict__ rp, const double *__restrict__ va,
                          const double *__restrict__ d, int64_t N, double *__restrict__ rowabs) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  double s = 0.0;
  for (int64_t q = rp[r]; q < rp[r + 1]; ++q) s += fabs(va[q]);
  rowabs[r] = s * d[r];
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

void launch_iteration(const IterArgs &a, cudaStream_t s) {
  k_spmv_res<<<a.ncta, kThreads, 0, s>>>(a);
  launch_proj(a, a.u, a.y, 1, s);
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

void launch_row_abs(const int64_t *rp, const double *va, const double *d, int64_t N,
                    double *rowabs, cudaStream_t s) {
  k_row_abs<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(rp, va, d, N, rowabs);
}

}  // namespace cimmino
