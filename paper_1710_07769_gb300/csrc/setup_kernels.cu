// Setup-stage kernels: input validation, row 2-norm scaling and permutation
// (Sections 2.1-2.2), transpose, C = A A^T SpGEMM (Section 2.3), extraction of the
// Gram blocks G_i (diagonal blocks of C) and their scatter into the tiled factor
// layout.
//
// Arithmetic that decides values (row norms, C entries) uses explicitly rounded
// multiply and add (no fused multiply-add), summing in increasing column index,
// so that scaled A and C are reproducible bit for bit run to run.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace cimmino {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n, int per_cta) {
  int64_t g = (n + per_cta - 1) / per_cta;
  return (unsigned)(g < 1 ? 1 : g);
}

// ---------------------------------------------------------------- validation
// flag bits: 1 = row_ptr not monotone / bad ends, 2 = column out of range,
// 4 = columns not strictly increasing
__global__ void k_validate_csr(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                               int64_t n, int64_t nnz, int32_t *flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(flag, 1);
  if (i >= n) return;
  int64_t a = rp[i], b = rp[i + 1];
  if (a > b || a < 0 || b > nnz) {
    atomicOr(flag, 1);
    return;
  }
  int32_t prev = -1;
  for (int64_t q = a; q < b; ++q) {
    int32_t c = ci[q];
    if (c < 0 || c >= n) atomicOr(flag, 2);
    if (c <= prev) atomicOr(flag, 4);
    prev = c;
  }
}

// ---------------------------------------------------------------- scan
// out[0] = 0, out[i+1] = counts[0] + ... + counts[i]; three passes over chunks of
// kScanChunk elements (chunk scan, scan of chunk totals, add-back).
constexpr int kScanPer = 8;
constexpr int kScanChunk = kThreads * kScanPer;

__global__ void k_scan_chunks(const int64_t *__restrict__ in, int64_t *__restrict__ out,
                              int64_t n, int64_t *__restrict__ totals) {
  __shared__ int64_t wsum[kThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanPer;
  int64_t v[kScanPer];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    int64_t idx = base + k;
    v[k] = idx < n ? in[idx] : 0;
    s += v[k];
  }
  // exclusive scan of per-thread sums across the CTA
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < kThreads / 32 ? wsum[lane] : 0;
    int64_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kThreads / 32) wsum[lane] = wi - w;  // exclusive warp offsets
    if (lane == kThreads / 32 - 1) totals[blockIdx.x] = wi;
  }
  __syncthreads();
  int64_t run = wsum[warp] + inc - s;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    run += v[k];
    int64_t idx = base + k;
    if (idx < n) out[idx + 1] = run;
  }
}

__global__ void k_scan_totals(int64_t *totals, int64_t nb) {
  // single CTA: exclusive scan of nb chunk totals, in place
  __shared__ int64_t carry;
  __shared__ int64_t wsum[kThreads / 32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t b0 = 0; b0 < nb; b0 += kThreads) {
    int64_t idx = b0 + threadIdx.x;
    int64_t v = idx < nb ? totals[idx] : 0;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    int64_t woff = 0;
    for (int w = 0; w < warp; ++w) woff += wsum[w];
    int64_t c = carry;
    if (idx < nb) totals[idx] = c + woff + inc - v;
    __syncthreads();
    if (threadIdx.x == kThreads - 1) carry = c + woff + inc;
    __syncthreads();
  }
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n,
                           const int64_t *__restrict__ totals) {
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  const int64_t add = totals[blockIdx.x];
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
  for (int k = threadIdx.x; k < kScanChunk; k += kThreads) {
    int64_t idx = base + k;
    if (idx < n) out[idx + 1] += add;
  }
}

// ---------------------------------------------------------------- scale + permute
__global__ void k_permuted_lengths(const int64_t *__restrict__ rp0, const int32_t *__restrict__ perm,
                                   int64_t N, int64_t *__restrict__ len) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  int64_t o = perm[r];
  len[r] = rp0[o + 1] - rp0[o];
}

// ---------------------------------------------------------------- equilibration
// Section 3.1: before the row 2-norm step, rows and columns are scaled so that the
// largest magnitude of every row and column tends to one.  One sweep takes the
// row maxima and the column maxima of the current matrix and divides entry (i, j)
// by sqrt(rmax_i) * sqrt(cmax_j) (an empty row or column keeps divisor 1).  Column
// maxima are combined with an integer atomicMax on the bit patterns, which order
// like the values for non-negative doubles, so the result does not depend on the
// order of the atomics.
__global__ void k_fill_one(double *__restrict__ a, double *__restrict__ b, int64_t N) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) a[i] = b[i] = 1.0;
}

__global__ void k_equil_max(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ v, int64_t N, double *__restrict__ rdiv,
                            unsigned long long *__restrict__ cmax) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  double m = 0.0;
  for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
    const double a = fabs(v[q]);
    if (a > m) m = a;
    atomicMax(&cmax[ci[q]], (unsigned long long)__double_as_longlong(a));
  }
  rdiv[r] = m > 0.0 ? __dsqrt_rn(m) : 1.0;
}

__global__ void k_equil_cols(unsigned long long *__restrict__ cmax, int64_t N,
                             double *__restrict__ cdiv, double *__restrict__ cs) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const double m = __longlong_as_double((long long)cmax[j]);
  cmax[j] = 0ull;  // ready for the next sweep
  const double dv = m > 0.0 ? __dsqrt_rn(m) : 1.0;
  cdiv[j] = dv;
  cs[j] = __dmul_rn(cs[j], dv);
}

__global__ void k_equil_apply(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              double *__restrict__ v, int64_t N, const double *__restrict__ rdiv,
                              const double *__restrict__ cdiv, double *__restrict__ rs) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const double dr = rdiv[r];
  for (int64_t q = rp[r]; q < rp[r + 1]; ++q) v[q] = __ddiv_rn(v[q], __dmul_rn(dr, cdiv[ci[q]]));
  rs[r] = __dmul_rn(rs[r], dr);
}

// Section 2.1: every row is divided by its 2-norm (so that the entries of
// A A^T are cosines); Section 2.2: permuted row r is original row perm[r].
// With equilibration, d[r] also carries the row's equilibration divisor rs.
__global__ void k_scale_permute(const int64_t *__restrict__ rp0, const int32_t *__restrict__ ci0,
                                const double *__restrict__ v0, const int32_t *__restrict__ perm,
                                const int64_t *__restrict__ rp, int64_t N,
                                int32_t *__restrict__ ci, double *__restrict__ va,
                                double *__restrict__ d, const double *__restrict__ rs,
                                int32_t *flag) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  int64_t o = perm[r];
  int64_t a = rp0[o], b = rp0[o + 1];
  double ss = 0.0;
  for (int64_t q = a; q < b; ++q) ss = __dadd_rn(ss, __dmul_rn(v0[q], v0[q]));
  double nr = sqrt(ss);
  if (!(nr > 0.0) || !isfinite(nr)) {
    atomicOr(flag, 1);
    nr = 1.0;
  }
  d[r] = rs ? __dmul_rn(nr, rs[o]) : nr;
  int64_t w = rp[r];
  for (int64_t q = a; q < b; ++q, ++w) {
    ci[w] = ci0[q];
    va[w] = __ddiv_rn(v0[q], nr);
  }
}

// ---------------------------------------------------------------- transpose
__global__ void k_col_count(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            int64_t N, unsigned long long *__restrict__ cnt) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  for (int64_t q = rp[r]; q < rp[r + 1]; ++q) atomicAdd(&cnt[ci[q]], 1ull);
}

__global__ void k_col_fill(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ va, int64_t N,
                           unsigned long long *__restrict__ cursor, int32_t *__restrict__ ri,
                           double *__restrict__ cv) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
    unsigned long long pos = atomicAdd(&cursor[ci[q]], 1ull);
    ri[pos] = (int32_t)r;
    cv[pos] = va[q];
  }
}

// rows inside a column end up in atomic order; sort them (insertion sort, columns
// of sparse matrices are short) so the transpose is deterministic.
__global__ void k_col_sort(const int64_t *__restrict__ cp, int64_t N, int32_t *__restrict__ ri,
                           double *__restrict__ cv) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  int64_t a = cp[k], b = cp[k + 1];
  for (int64_t q = a + 1; q < b; ++q) {
    int32_t key = ri[q];
    double val = cv[q];
    int64_t t = q - 1;
    while (t >= a && ri[t] > key) {
      ri[t + 1] = ri[t];
      cv[t + 1] = cv[t];
      --t;
    }
    ri[t + 1] = key;
    cv[t + 1] = val;
  }
}

// ---------------------------------------------------------------- SpGEMM C = A A^T
// Row i of C: the candidate set is the union, over the columns k of row i, of the
// rows of column k.  A group (a warp, or a whole CTA for long rows) gathers the
// candidates into shared memory, sorts them (bitonic) and keeps the distinct ones.
// Values follow the definition c_ij = sum_k a_ik a_jk, evaluated by merging the two
// sorted rows in increasing k -- the same order as Gustavson's accumulation.

// Rows of column k of A (sorted ascending in the transpose) that fall in [lo, hi): the
// candidates of a row whose output is restricted to its own block's rows.
__device__ __forceinline__ void col_window(const int32_t *__restrict__ ri, int64_t &s0,
                                           int64_t &e0, int32_t lo, int32_t hi) {
  if (lo <= 0 && hi == INT32_MAX) return;
  int64_t a = s0, b = e0;
  while (a < b) {  // first row >= lo
    const int64_t m = (a + b) >> 1;
    if (ri[m] < lo) a = m + 1; else b = m;
  }
  int64_t c = a, d = e0;
  while (c < d) {  // first row >= hi
    const int64_t m = (c + d) >> 1;
    if (ri[m] < hi) c = m + 1; else d = m;
  }
  s0 = a;
  e0 = c;
}

// The output window of row i: its block's rows when blk is given, else every row.
__device__ __forceinline__ void row_window(const BlockDesc *__restrict__ blk,
                                           const int32_t *__restrict__ rowblk, int64_t i,
                                           int32_t &lo, int32_t &hi) {
  lo = 0;
  hi = INT32_MAX;
  if (blk) {
    const BlockDesc B = blk[rowblk[i]];
    lo = (int32_t)B.row0;
    hi = (int32_t)(B.row0 + B.m);
  }
}

template <int G>
__device__ __forceinline__ void group_sync() {
  if (G == 32)
    __syncwarp();
  else
    __syncthreads();
}

template <int G>
__device__ int gather_candidates(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                 const int64_t *__restrict__ cp, const int32_t *__restrict__ ri,
                                 int64_t i, int32_t *buf, int cap, int gt, int32_t wlo,
                                 int32_t whi) {
  int U = 0;
  for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
    int32_t k = ci[q];
    int64_t s0 = cp[k], e0 = cp[k + 1];
    col_window(ri, s0, e0, wlo, whi);
    int len = (int)(e0 - s0);
    for (int t = gt; t < len; t += G)
      if (U + t < cap) buf[U + t] = ri[s0 + t];
    U += len;
  }
  group_sync<G>();
  return U;
}

// Warp gather of the candidates of row i when the row has at most 32 entries: lane q looks
// up column j_q's range in the transpose (all lanes at once), a warp scan gives each
// column's offset in the candidate list, and then every lane fetches its candidates (and,
// with val, the products a_ij a_rj) independently, so the row costs a few dependent loads
// instead of a chain per column.  Candidates are in column order, rows increasing within a
// column, the order of the serial gather.  Returns the total (entries beyond cap are not
// written); key/val (optional): 64-bit (row << 32 | position of j in row i) and products.
struct WarpCols {
  int32_t off[32];
  int64_t start[32];
  double a[32];
};

__device__ int gather_warp(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ va, const int64_t *__restrict__ cp,
                           const int32_t *__restrict__ ri, const double *__restrict__ cv,
                           int64_t i, WarpCols &wc, int32_t *rows, uint64_t *key, double *val,
                           int cap, int lane, int32_t wlo, int32_t whi) {
  const int64_t q0 = rp[i];
  const int nq = (int)(rp[i + 1] - q0);
  int len = 0;
  if (lane < nq) {
    const int32_t j = ci[q0 + lane];
    int64_t s0 = cp[j], e0 = cp[j + 1];
    col_window(ri, s0, e0, wlo, whi);
    len = (int)(e0 - s0);
    wc.start[lane] = s0;
    if (val) wc.a[lane] = va[q0 + lane];
  }
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane < nq) wc.off[lane] = incl - len;
  const int U = __shfl_sync(0xffffffffu, incl, 31);
  __syncwarp();
  const int lim = U < cap ? U : cap;
  for (int t = lane; t < lim; t += 32) {
    int lo = 0, hi = nq - 1;  // last column whose offset is <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (wc.off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int64_t e = wc.start[lo] + (t - wc.off[lo]);
    const int32_t r = ri[e];
    if (rows) rows[t] = r;
    if (key) key[t] = ((uint64_t)(uint32_t)r << 32) | (uint32_t)lo;
    if (val) val[t] = __dmul_rn(wc.a[lo], cv[e]);
  }
  __syncwarp();
  return U;
}

// Number of distinct candidate rows of row i (at most 32 entries) when there are at most
// kHashCands candidates: a shared-memory hash set of kHashSlots slots (linear probing,
// atomicCAS), no sort.  Returns -1 when the row has more candidates.
constexpr int kHashSlots = kSpgemmWarpCap;  // the warp's 4 KB buffer
constexpr int kHashCands = kHashSlots / 2;

__device__ int count_unique_warp(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                 const int64_t *__restrict__ cp, const int32_t *__restrict__ ri,
                                 int64_t i, WarpCols &wc, int32_t *table, int lane,
                                 int32_t wlo, int32_t whi) {
  const int64_t q0 = rp[i];
  const int nq = (int)(rp[i + 1] - q0);
  int len = 0;
  if (lane < nq) {
    const int32_t j = ci[q0 + lane];
    int64_t s0 = cp[j], e0 = cp[j + 1];
    col_window(ri, s0, e0, wlo, whi);
    len = (int)(e0 - s0);
    wc.start[lane] = s0;
  }
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane < nq) wc.off[lane] = incl - len;
  const int U = __shfl_sync(0xffffffffu, incl, 31);
  if (U > kHashCands) return -1;
  for (int t = lane; t < kHashSlots; t += 32) table[t] = -1;
  __syncwarp();
  int mine = 0;
  for (int t = lane; t < U; t += 32) {
    int lo = 0, hi = nq - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (wc.off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int32_t r = ri[wc.start[lo] + (t - wc.off[lo])];
    uint32_t h = ((uint32_t)r * 2654435761u) >> 22;  // 10 bits: kHashSlots = 1024
    for (int probe = 0; probe < kHashSlots; ++probe) {
      const int32_t prev = atomicCAS(&table[h], -1, r);
      if (prev == -1) {
        ++mine;
        break;
      }
      if (prev == r) break;
      h = (h + 1) & (kHashSlots - 1);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  __syncwarp();
  return mine;
}
static_assert(kHashSlots == 1024, "the hash takes 10 bits");

template <int G>
__device__ void bitonic_sort(int32_t *buf, int U, int gt) {
  int P = 1;
  while (P < U) P <<= 1;
  for (int t = U + gt; t < P; t += G) buf[t] = 0x7fffffff;
  group_sync<G>();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = gt; t < P; t += G) {
        int ixj = t ^ j;
        if (ixj > t) {
          int32_t a = buf[t], b = buf[ixj];
          bool up = (t & k) == 0;
          if ((a > b) == up) {
            buf[t] = b;
            buf[ixj] = a;
          }
        }
      }
      group_sync<G>();
    }
  }
}

// in-place compaction of the distinct values of sorted buf[0..U); returns count
template <int G>
__device__ int unique_compact(int32_t *buf, int U, int gt) {
  if (G == 32) {
    int total = 0;
    for (int base = 0; base < U; base += 32) {
      int t = base + gt;
      int32_t v = t < U ? buf[t] : 0;
      bool keep = t < U && (t == 0 || buf[t - 1] != v);
      unsigned m = __ballot_sync(0xffffffffu, keep);
      int pos = total + __popc(m & ((1u << gt) - 1u));
      __syncwarp();
      if (keep) buf[pos] = v;  // pos <= t: never overwrites an unread later entry
      __syncwarp();
      total += __popc(m);
    }
    return total;
  } else {
    __shared__ int s_total;
    if (gt == 0) {
      int w = 0;
      for (int t = 0; t < U; ++t)
        if (t == 0 || buf[t] != buf[w - 1]) buf[w++] = buf[t];
      s_total = w;
    }
    __syncthreads();
    int r = s_total;
    __syncthreads();
    return r;
  }
}

__device__ __forceinline__ double row_dot(const int64_t *__restrict__ rp,
                                          const int32_t *__restrict__ ci,
                                          const double *__restrict__ va, int64_t i, int64_t j) {
  int64_t qa = rp[i], ea = rp[i + 1], qb = rp[j], eb = rp[j + 1];
  double acc = 0.0;
  bool first = true;
  while (qa < ea && qb < eb) {
    int32_t ka = ci[qa], kb = ci[qb];
    if (ka == kb) {
      double prod = __dmul_rn(va[qa], va[qb]);
      acc = first ? prod : __dadd_rn(acc, prod);
      first = false;
      ++qa;
      ++qb;
    } else if (ka < kb) {
      ++qa;
    } else {
      ++qb;
    }
  }
  return acc;
}

constexpr int kSpgemmWarps = 8;

// count pass, one warp per row; rows with more than kSpgemmWarpCap candidates are
// appended to an overflow list (handled by the CTA-per-row variant).
__global__ void __launch_bounds__(kSpgemmWarps * 32)
    k_spgemm_count_warp(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                        const int64_t *__restrict__ cp, const int32_t *__restrict__ ri,
                        int64_t N, int64_t *__restrict__ cnt, int32_t *__restrict__ ovf_list,
                        int32_t *__restrict__ ovf_n, const BlockDesc *__restrict__ blk,
                        const int32_t *__restrict__ rowblk) {
  __shared__ int32_t sbuf[kSpgemmWarps][kSpgemmWarpCap];
  __shared__ WarpCols scols[kSpgemmWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t i = (int64_t)blockIdx.x * kSpgemmWarps + warp;
  if (i >= N) return;
  int32_t wlo, whi;
  row_window(blk, rowblk, i, wlo, whi);
  int32_t *buf = sbuf[warp];
  if (rp[i + 1] - rp[i] <= 32) {
    const int u = count_unique_warp(rp, ci, cp, ri, i, scols[warp], buf, lane, wlo, whi);
    if (u >= 0) {
      if (lane == 0) cnt[i] = u;
      return;
    }
  }
  const int U = rp[i + 1] - rp[i] <= 32
                    ? gather_warp(rp, ci, nullptr, cp, ri, nullptr, i, scols[warp], buf, nullptr,
                                  nullptr, kSpgemmWarpCap, lane, wlo, whi)
                    : gather_candidates<32>(rp, ci, cp, ri, i, buf, kSpgemmWarpCap, lane, wlo,
                                            whi);
  if (U > kSpgemmWarpCap) {
    if (lane == 0) {
      int slot = atomicAdd(ovf_n, 1);
      ovf_list[slot] = (int32_t)i;
      cnt[i] = 0;
    }
    return;
  }
  bitonic_sort<32>(buf, U, lane);
  int u = unique_compact<32>(buf, U, lane);
  if (lane == 0) cnt[i] = u;
}

// Rows of C with at most kFillFast candidates are filled by Gustavson's scheme: every
// (candidate row r, column j) pair of row i carries its product a_ij a_rj, the pairs are
// sorted by (r, position of j in row i), and each run of equal r is summed in increasing j,
// the order of the row-wise definition (explicitly rounded products and sums, so the values
// are those of a sequential loop).  Longer rows take the dot-product path below.
constexpr int kFillFast = kSpgemmWarpCap / 4;  // 16-byte pairs in the warp's 4 KB buffer
// rows with at most kHashFill candidates use a hash table (rows, products, table keys and
// values: 24 bytes per candidate in the same 4 KB buffer)
constexpr int kHashFillBits = 7;
constexpr int kHashFill = 1 << kHashFillBits;
static_assert(24 * kHashFill <= 4 * kSpgemmWarpCap, "hash fill inside the warp buffer");

__device__ void bitonic_sort_kv(uint64_t *key, double *val, int U, int lane) {
  int P = 1;
  while (P < U) P <<= 1;
  for (int t = U + lane; t < P; t += 32) key[t] = ~0ull;
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < P; t += 32) {
        const int ixj = t ^ j;
        if (ixj > t) {
          const uint64_t a = key[t], b = key[ixj];
          const bool up = (t & k) == 0;
          if ((a > b) == up) {
            key[t] = b;
            key[ixj] = a;
            const double va = val[t];
            val[t] = val[ixj];
            val[ixj] = va;
          }
        }
      }
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(kSpgemmWarps * 32)
    k_spgemm_fill_warp(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                       const double *__restrict__ va, const int64_t *__restrict__ cp,
                       const int32_t *__restrict__ ri, const double *__restrict__ cv, int64_t N,
                       const int64_t *__restrict__ crp, int32_t *__restrict__ cci,
                       double *__restrict__ ccv, const BlockDesc *__restrict__ blk,
                       const int32_t *__restrict__ rowblk) {
  __shared__ __align__(16) int32_t sbuf[kSpgemmWarps][kSpgemmWarpCap];
  __shared__ WarpCols scols[kSpgemmWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t i = (int64_t)blockIdx.x * kSpgemmWarps + warp;
  if (i >= N) return;
  int32_t wlo, whi;
  row_window(blk, rowblk, i, wlo, whi);
  int32_t *buf = sbuf[warp];
  const int nq = (int)(rp[i + 1] - rp[i]);
  uint64_t *key = reinterpret_cast<uint64_t *>(buf);
  double *val = reinterpret_cast<double *>(buf) + kFillFast;
  // rows of at most 32 entries whose candidates fit the sort buffer: Gustavson's scheme
  if (nq <= 32) {
    // up to kHashFill candidates: accumulate a_ij a_rj per candidate row r in a shared hash
    // table, one column j after the other (so every r sums in increasing j), then place
    // each distinct r at its rank among the row's distinct candidates (no sort)
    int32_t *crow = buf;                                               // [kHashFill]
    double *cval = reinterpret_cast<double *>(buf + kHashFill);        // [kHashFill]
    int32_t *hk = buf + 3 * kHashFill;                                 // [kHashFill]
    double *hv = reinterpret_cast<double *>(buf + 4 * kHashFill);      // [kHashFill]
    const int Uh = gather_warp(rp, ci, va, cp, ri, cv, i, scols[warp], crow, nullptr, cval,
                               kHashFill, lane, wlo, whi);
    if (Uh <= kHashFill) {
      for (int t = lane; t < kHashFill; t += 32) hk[t] = -1;
      __syncwarp();
      const WarpCols &wc = scols[warp];
      for (int q = 0; q < nq; ++q) {
        const int t1 = q + 1 < nq ? wc.off[q + 1] : Uh;
        for (int t = wc.off[q] + lane; t < t1; t += 32) {
          const int32_t r = crow[t];
          const double pr = cval[t];
          uint32_t h = ((uint32_t)r * 2654435761u) >> (32 - kHashFillBits);
          for (int probe = 0; probe < kHashFill; ++probe) {
            const int32_t prev = atomicCAS(&hk[h], -1, r);
            if (prev == -1) {
              hv[h] = pr;
              break;
            }
            if (prev == r) {
              hv[h] = __dadd_rn(hv[h], pr);
              break;
            }
            h = (h + 1) & (kHashFill - 1);
          }
        }
        __syncwarp();
      }
      int total = 0;
      for (int b0 = 0; b0 < kHashFill; b0 += 32) {
        const int sl = b0 + lane;
        const bool occ = hk[sl] >= 0;
        const unsigned m = __ballot_sync(0xffffffffu, occ);
        if (occ) {
          const int pos = total + __popc(m & ((1u << lane) - 1u));
          crow[pos] = hk[sl];
          cval[pos] = hv[sl];
        }
        total += __popc(m);
      }
      __syncwarp();
      const int64_t w = crp[i];
      for (int e = lane; e < total; e += 32) {
        const int32_t r = crow[e];
        int rank = 0;
        for (int m = 0; m < total; ++m) rank += crow[m] < r;
        cci[w + rank] = r;
        ccv[w + rank] = cval[e];
      }
      return;
    }
  }
  const int U = nq <= 32 ? gather_warp(rp, ci, va, cp, ri, cv, i, scols[warp], nullptr, key,
                                       val, kFillFast, lane, wlo, whi)
                         : kFillFast + 1;
  if (U <= kFillFast) {
    bitonic_sort_kv(key, val, U, lane);
    const int64_t w = crp[i];
    int total = 0;
    for (int b0 = 0; b0 < U; b0 += 32) {
      const int t = b0 + lane;
      const bool head = t < U && (t == 0 || (key[t] >> 32) != (key[t - 1] >> 32));
      const unsigned m = __ballot_sync(0xffffffffu, head);
      if (head) {
        const uint64_t r = key[t] >> 32;
        double acc = val[t];
        for (int u = t + 1; u < U && (key[u] >> 32) == r; ++u) acc = __dadd_rn(acc, val[u]);
        const int pos = total + __popc(m & ((1u << lane) - 1u));
        cci[w + pos] = (int32_t)r;
        ccv[w + pos] = acc;
      }
      total += __popc(m);
    }
    return;
  }
  const int Ul = gather_candidates<32>(rp, ci, cp, ri, i, buf, kSpgemmWarpCap, lane, wlo, whi);
  if (Ul > kSpgemmWarpCap) return;  // CTA variant fills this row
  bitonic_sort<32>(buf, Ul, lane);
  int u = unique_compact<32>(buf, Ul, lane);
  int64_t w = crp[i];
  for (int t = lane; t < u; t += 32) {
    int32_t j = buf[t];
    cci[w + t] = j;
    ccv[w + t] = row_dot(rp, ci, va, i, j);
  }
}

__global__ void k_spgemm_cta(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const double *__restrict__ va, const int64_t *__restrict__ cp,
                             const int32_t *__restrict__ ri, const int32_t *__restrict__ ovf_list,
                             int64_t *__restrict__ cnt, const int64_t *__restrict__ crp,
                             int32_t *__restrict__ cci, double *__restrict__ ccv,
                             int32_t *flag, const BlockDesc *__restrict__ blk,
                             const int32_t *__restrict__ rowblk) {
  extern __shared__ int32_t dbuf[];
  const int64_t i = ovf_list[blockIdx.x];
  int32_t wlo, whi;
  row_window(blk, rowblk, i, wlo, whi);
  int U = gather_candidates<kThreads>(rp, ci, cp, ri, i, dbuf, kSpgemmCtaCap, threadIdx.x, wlo,
                                      whi);
  if (U > kSpgemmCtaCap) {
    if (threadIdx.x == 0) atomicOr(flag, 8);
    return;
  }
  bitonic_sort<kThreads>(dbuf, U, threadIdx.x);
  int u = unique_compact<kThreads>(dbuf, U, threadIdx.x);
  if (crp == nullptr) {
    if (threadIdx.x == 0) cnt[i] = u;
    return;
  }
  int64_t w = crp[i];
  for (int t = threadIdx.x; t < u; t += kThreads) {
    int32_t j = dbuf[t];
    cci[w + t] = j;
    ccv[w + t] = row_dot(rp, ci, va, i, j);
  }
}

// ---------------------------------------------------------------- block-diagonal part of C
__global__ void k_row_block_ids(const BlockDesc *__restrict__ blk, int32_t nblk,
                                int32_t *__restrict__ rowblk) {
  int b = blockIdx.x;
  if (b >= nblk) return;
  BlockDesc B = blk[b];
  for (int r = threadIdx.x; r < B.m; r += blockDim.x) rowblk[B.row0 + r] = b;
}

__global__ void k_bd_count(const int64_t *__restrict__ crp, const int32_t *__restrict__ cci,
                           const BlockDesc *__restrict__ blk, const int32_t *__restrict__ rowblk,
                           int64_t N, int64_t *__restrict__ cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  BlockDesc B = blk[rowblk[i]];
  int64_t lo = B.row0, hi = B.row0 + B.m;
  int64_t c = 0;
  for (int64_t q = crp[i]; q < crp[i + 1]; ++q) {
    int64_t j = cci[q];
    c += (j >= lo && j < hi);
  }
  cnt[i] = c;
}

// G_i = C restricted to block i (both triangles, local column indices); rowmin[i]
// = first local column of the row, the left end of its envelope.
__global__ void k_bd_fill(const int64_t *__restrict__ crp, const int32_t *__restrict__ cci,
                          const double *__restrict__ ccv, const BlockDesc *__restrict__ blk,
                          const int32_t *__restrict__ rowblk, int64_t N,
                          const int64_t *__restrict__ brp, int32_t *__restrict__ bci,
                          double *__restrict__ bcv, int32_t *__restrict__ rowmin) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  BlockDesc B = blk[rowblk[i]];
  int64_t lo = B.row0, hi = B.row0 + B.m;
  int64_t w = brp[i];
  int32_t mn = (int32_t)(i - lo);
  for (int64_t q = crp[i]; q < crp[i + 1]; ++q) {
    int64_t j = cci[q];
    if (j >= lo && j < hi) {
      int32_t lj = (int32_t)(j - lo);
      bci[w] = lj;
      bcv[w] = ccv[q];
      ++w;
      if (lj < mn) mn = lj;
    }
  }
  rowmin[i] = mn;
}

// Rows of C restricted to their own block (the Gram blocks, computed directly): global
// columns become block-local ones and rowmin[i] gets the row's first local column.
__global__ void k_bd_local(const int64_t *__restrict__ brp, int32_t *__restrict__ bci,
                           const BlockDesc *__restrict__ blk, const int32_t *__restrict__ rowblk,
                           int64_t N, int32_t *__restrict__ rowmin) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t lo = blk[rowblk[i]].row0;
  int32_t mn = (int32_t)(i - lo);
  for (int64_t q = brp[i]; q < brp[i + 1]; ++q) {
    const int32_t lj = (int32_t)(bci[q] - lo);
    bci[q] = lj;
    if (lj < mn) mn = lj;
  }
  rowmin[i] = mn;
}

// J0 of every tile row: the smallest tile column touched by the envelope of the
// rows of the tile row (0 for the dense layout).
__global__ void k_tile_j0(const BlockDesc *__restrict__ blk, int32_t nblk,
                          const int32_t *__restrict__ rowmin, int dense,
                          int32_t *__restrict__ j0) {
  int b = blockIdx.x;
  if (b >= nblk) return;
  BlockDesc B = blk[b];
  for (int I = threadIdx.x; I < B.nt; I += blockDim.x) {
    int v = I;
    if (!dense) {
      int r1 = min((I + 1) * kTile, B.m);
      for (int r = I * kTile; r < r1; ++r) v = min(v, rowmin[B.row0 + r] / kTile);
    } else {
      v = 0;
    }
    j0[B.trow0 + I] = v;
  }
}

// Sliced-ELL copy of the Gram blocks (slices of 32 consecutive rows of a block,
// entries stored [k][lane] so that a warp reads 32 consecutive values), used by the
// FP64 refinement residual res = u - G_i y.  Width of a slice = its longest row.
__global__ void k_sell_width(const BlockDesc *__restrict__ blk, int32_t nblk,
                             const int64_t *__restrict__ brp, int64_t *__restrict__ cnt) {
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const BlockDesc B = blk[b];
  const int ns = (B.m + 31) / 32;
  for (int sl = threadIdx.x; sl < ns; sl += blockDim.x) {
    int64_t w = 0;
    for (int l = 0; l < 32; ++l) {
      const int r = sl * 32 + l;
      if (r < B.m) w = max(w, brp[B.row0 + r + 1] - brp[B.row0 + r]);
    }
    cnt[B.slice0 + sl] = 32 * w;
  }
}

__global__ void k_sell_fill(const BlockDesc *__restrict__ blk, int32_t nblk,
                            const int64_t *__restrict__ brp, const int32_t *__restrict__ bci,
                            const double *__restrict__ bcv, const int64_t *__restrict__ soff,
                            int16_t *__restrict__ scol, double *__restrict__ sval) {
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const BlockDesc B = blk[b];
  const int ns = (B.m + 31) / 32;
  for (int r = threadIdx.x; r < ns * 32; r += blockDim.x) {
    const int sl = B.slice0 + r / 32, l = r % 32;
    const int64_t o = soff[sl];
    const int w = (int)((soff[sl + 1] - o) / 32);
    const int64_t p0 = r < B.m ? brp[B.row0 + r] : 0;
    const int len = r < B.m ? (int)(brp[B.row0 + r + 1] - p0) : 0;
    for (int k = 0; k < w; ++k) {
      const bool real = k < len;
      scol[o + (int64_t)k * 32 + l] = real ? (int16_t)bci[p0 + k] : (int16_t)0;
      sval[o + (int64_t)k * 32 + l] = real ? bcv[p0 + k] : 0.0;
    }
  }
}

// Sliced-ELL copy of a CSR matrix (used for A and for A^T): slice k covers rows
// srow0[k] .. srow0[k] + srows[k] - 1 (at most 32, never straddling systems); entry k
// of lane l sits at off + 32 k + l.  Padding entries point at the slice's first row
// with value 0, so they read a valid element and add nothing.
// Rows of one CTA-table chunk in order of decreasing length (ties: increasing row), so that
// the 32-row slices of a sliced-ELL copy hold rows of similar length and pad little:
// ord[row0 + rank] = row.  One CTA (kVecRows threads) per chunk.
__global__ void __launch_bounds__(kVecRows)
    k_chunk_order(const int64_t *__restrict__ ptr, const CtaDesc *__restrict__ cta,
                  int32_t *__restrict__ ord) {
  __shared__ int64_t len[kVecRows];
  const CtaDesc C = cta[blockIdx.x];
  const int t = threadIdx.x;
  const int64_t r = C.row0 + t;
  len[t] = t < C.rows ? ptr[r + 1] - ptr[r] : -1;
  __syncthreads();
  if (t >= C.rows) return;
  const int64_t mine = len[t];
  int rank = 0;
  for (int u = 0; u < C.rows; ++u) rank += len[u] > mine || (len[u] == mine && u < t);
  ord[C.row0 + rank] = (int32_t)r;
}

// rmap (optional): the row in position srow0 + l of the copy
__global__ void k_sell_rows_width(const int64_t *__restrict__ ptr, const int64_t *__restrict__ srow0,
                                  const int32_t *__restrict__ srows, int32_t nslice,
                                  const int32_t *__restrict__ rmap, int64_t *__restrict__ cnt) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nslice) return;
  int64_t w = 0;
  for (int l = 0; l < srows[k]; ++l) {
    const int64_t r = rmap ? rmap[srow0[k] + l] : srow0[k] + l;
    w = max(w, ptr[r + 1] - ptr[r]);
  }
  cnt[k] = 32 * w;
}

__global__ void k_sell_rows_fill(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                 const double *__restrict__ val, const int64_t *__restrict__ srow0,
                                 const int32_t *__restrict__ srows, int32_t nslice,
                                 const int32_t *__restrict__ rmap,
                                 const int64_t *__restrict__ off, int32_t *__restrict__ ocol,
                                 double *__restrict__ oval) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = (int)(g >> 5), l = (int)(g & 31);
  if (k >= nslice) return;
  const int64_t o = off[k];
  const int w = (int)((off[k + 1] - o) >> 5);
  const bool real = l < srows[k];
  const int64_t r = real && rmap ? rmap[srow0[k] + l] : srow0[k] + l;
  const int64_t p0 = real ? ptr[r] : 0;
  const int len = real ? (int)(ptr[r + 1] - p0) : 0;
  for (int e = 0; e < w; ++e) {
    const bool in = e < len;
    ocol[o + 32 * (int64_t)e + l] = in ? idx[p0 + e] : (int32_t)srow0[k];
    oval[o + 32 * (int64_t)e + l] = in ? val[p0 + e] : 0.0;
  }
}

// Write the lower triangle of G_b into the tiles of its factor (zeroing the tile
// row first); padded rows beyond m get a unit diagonal.
template <typename W>
__global__ void k_gram_scatter(const BlockDesc *__restrict__ blk, const int32_t *__restrict__ blist,
                               const TileRow *__restrict__ trow, const int64_t *__restrict__ brp,
                               const int32_t *__restrict__ bci, const double *__restrict__ bcv,
                               W *__restrict__ fac) {
  const int b = blist[blockIdx.x];
  const BlockDesc B = blk[b];
  const int mp = B.nt * kTile;
  // the tiles were zeroed by one memset of the whole factor array before the launch
  for (int r = threadIdx.x; r < mp; r += blockDim.x) {
    const int I = r / kTile, rr = r % kTile;
    const TileRow T = trow[B.trow0 + I];
    W *rowbase = fac + T.off + (int64_t)rr * kTile;
    if (r >= B.m) {
      rowbase[(int64_t)(I - T.j0) * kTile * kTile + rr] = W(1);
      continue;
    }
    const int64_t gi = B.row0 + r;
    for (int64_t q = brp[gi]; q < brp[gi + 1]; ++q) {
      int j = bci[q];
      if (j > r) break;  // columns sorted: only the lower triangle is stored
      int J = j / kTile;
      rowbase[(int64_t)(J - T.j0) * kTile * kTile + (j % kTile)] = W(bcv[q]);
    }
  }
}

}  // namespace

// perm is a permutation of 0..n-1: every value in range and taken once (seen: n zeros)
__global__ void k_check_perm(const int32_t *__restrict__ perm, int64_t n, int32_t *seen,
                             int32_t *flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t v = perm[i];
  if (v < 0 || v >= n || atomicAdd(&seen[v], 1) != 0) atomicOr(flag, 1);
}

// ================================================================ launchers
void launch_validate_csr(const int64_t *rp, const int32_t *ci, int64_t n, int64_t nnz,
                         int32_t *flag, cudaStream_t s) {
  k_validate_csr<<<grid_for(n + 1, kThreads), kThreads, 0, s>>>(rp, ci, n, nnz, flag);
}

void launch_check_perm(const int32_t *perm, int64_t n, int32_t *seen, int32_t *flag,
                       cudaStream_t s) {
  k_check_perm<<<grid_for(n, kThreads), kThreads, 0, s>>>(perm, n, seen, flag);
}

int64_t scan_tmp_len(int64_t n) { return (n + kScanChunk - 1) / kScanChunk + 1; }

void launch_scan_counts(const int64_t *counts, int64_t *out, int64_t n, int64_t *tmp,
                        int64_t tmp_len, cudaStream_t s) {
  int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  if (nb < 1) nb = 1;
  (void)tmp_len;
  k_scan_chunks<<<(unsigned)nb, kThreads, 0, s>>>(counts, out, n, tmp);
  k_scan_totals<<<1, kThreads, 0, s>>>(tmp, nb);
  k_scan_add<<<(unsigned)nb, kThreads, 0, s>>>(out, n, tmp);
}

void launch_permuted_lengths(const int64_t *rp0, const int32_t *perm, int64_t N, int64_t *len,
                             cudaStream_t s) {
  k_permuted_lengths<<<grid_for(N, kThreads), kThreads, 0, s>>>(rp0, perm, N, len);
}

void launch_scale_permute(const int64_t *rp0, const int32_t *ci0, const double *v0,
                          const int32_t *perm, const int64_t *rp, int64_t N, int32_t *ci,
                          double *va, double *d, const double *rs, int32_t *flag,
                          cudaStream_t s) {
  k_scale_permute<<<grid_for(N, kThreads), kThreads, 0, s>>>(rp0, ci0, v0, perm, rp, N, ci, va,
                                                             d, rs, flag);
}

void launch_equilibrate(const int64_t *rp, const int32_t *ci, double *v, int64_t N,
                        int32_t sweeps, double *rs, double *cs, double *work, cudaStream_t s) {
  double *rdiv = work, *cdiv = work + N;
  unsigned long long *cmax = reinterpret_cast<unsigned long long *>(work + 2 * N);
  k_fill_one<<<grid_for(N, kThreads), kThreads, 0, s>>>(rs, cs, N);
  cudaMemsetAsync(cmax, 0, sizeof(unsigned long long) * N, s);
  for (int32_t t = 0; t < sweeps; ++t) {
    k_equil_max<<<grid_for(N, kThreads), kThreads, 0, s>>>(rp, ci, v, N, rdiv, cmax);
    k_equil_cols<<<grid_for(N, kThreads), kThreads, 0, s>>>(cmax, N, cdiv, cs);
    k_equil_apply<<<grid_for(N, kThreads), kThreads, 0, s>>>(rp, ci, v, N, rdiv, cdiv, rs);
  }
}

void launch_transpose(const int64_t *rp, const int32_t *ci, const double *va, int64_t N,
                      int64_t nnz, int64_t *cp, int32_t *ri, double *cv, int64_t *work,
                      int64_t *tmp, int64_t tmp_len, cudaStream_t s) {
  // work: 2*N int64 (column counts, then fill cursors)
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(work);
  unsigned long long *cur = cnt + N;
  cudaMemsetAsync(cnt, 0, sizeof(int64_t) * N, s);
  k_col_count<<<grid_for(N, kThreads), kThreads, 0, s>>>(rp, ci, N, cnt);
  launch_scan_counts(reinterpret_cast<int64_t *>(cnt), cp, N, tmp, tmp_len, s);
  cudaMemcpyAsync(cur, cp, sizeof(int64_t) * N, cudaMemcpyDeviceToDevice, s);
  k_col_fill<<<grid_for(N, kThreads), kThreads, 0, s>>>(rp, ci, va, N, cur, ri, cv);
  k_col_sort<<<grid_for(N, kThreads), kThreads, 0, s>>>(cp, N, ri, cv);
  (void)nnz;
}

void spgemm_count(const int64_t *rp, const int32_t *ci, const int64_t *cp, const int32_t *ri,
                  int64_t N, int64_t *cnt, int32_t *ovf, int32_t *ovf_n, cudaStream_t s,
                  const BlockDesc *blk, const int32_t *rowblk) {
  cudaMemsetAsync(ovf_n, 0, sizeof(int32_t), s);
  k_spgemm_count_warp<<<grid_for(N, kSpgemmWarps), kSpgemmWarps * 32, 0, s>>>(
      rp, ci, cp, ri, N, cnt, ovf, ovf_n, blk, rowblk);
}

void spgemm_overflow(const int64_t *rp, const int32_t *ci, const double *va, const int64_t *cp,
                     const int32_t *ri, const int32_t *ovf, int32_t novf, int64_t *cnt,
                     const int64_t *crp, int32_t *cci, double *ccv, int32_t *flag,
                     cudaStream_t s, const BlockDesc *blk, const int32_t *rowblk) {
  if (novf <= 0) return;
  size_t smem = sizeof(int32_t) * kSpgemmCtaCap;
  k_spgemm_cta<<<(unsigned)novf, kThreads, smem, s>>>(rp, ci, va, cp, ri, ovf, cnt, crp, cci,
                                                      ccv, flag, blk, rowblk);
}

void spgemm_fill(const int64_t *rp, const int32_t *ci, const double *va, const int64_t *cp,
                 const int32_t *ri, const double *cv, int64_t N, const int64_t *crp,
                 int32_t *cci, double *ccv, cudaStream_t s, const BlockDesc *blk,
                 const int32_t *rowblk) {
  k_spgemm_fill_warp<<<grid_for(N, kSpgemmWarps), kSpgemmWarps * 32, 0, s>>>(
      rp, ci, va, cp, ri, cv, N, crp, cci, ccv, blk, rowblk);
}

void launch_row_block_ids(const BlockDesc *blk, int32_t nblk, int32_t *rowblk, cudaStream_t s) {
  if (nblk > 0) k_row_block_ids<<<(unsigned)nblk, kThreads, 0, s>>>(blk, nblk, rowblk);
}

void bd_count(const int64_t *crp, const int32_t *cci, const BlockDesc *blk, const int32_t *rowblk,
              int64_t N, int64_t *cnt, cudaStream_t s) {
  k_bd_count<<<grid_for(N, kThreads), kThreads, 0, s>>>(crp, cci, blk, rowblk, N, cnt);
}

void bd_localize(const int64_t *brp, int32_t *bci, const BlockDesc *blk, const int32_t *rowblk,
                 int64_t N, int32_t *rowmin, cudaStream_t s) {
  k_bd_local<<<grid_for(N, kThreads), kThreads, 0, s>>>(brp, bci, blk, rowblk, N, rowmin);
}

void bd_fill(const int64_t *crp, const int32_t *cci, const double *ccv, const BlockDesc *blk,
             const int32_t *rowblk, int64_t N, const int64_t *brp, int32_t *bci, double *bcv,
             int32_t *rowmin, cudaStream_t s) {
  k_bd_fill<<<grid_for(N, kThreads), kThreads, 0, s>>>(crp, cci, ccv, blk, rowblk, N, brp, bci,
                                                       bcv, rowmin);
}

void launch_tile_j0(const BlockDesc *blk, int32_t nblk, const int32_t *rowmin, int dense,
                    int32_t *j0, cudaStream_t s) {
  if (nblk > 0) k_tile_j0<<<(unsigned)nblk, 64, 0, s>>>(blk, nblk, rowmin, dense, j0);
}

void sell_width(const BlockDesc *blk, int32_t nblk, const int64_t *brp, int64_t *cnt,
                cudaStream_t s) {
  if (nblk > 0) k_sell_width<<<(unsigned)nblk, 64, 0, s>>>(blk, nblk, brp, cnt);
}

void sell_fill(const BlockDesc *blk, int32_t nblk, const int64_t *brp, const int32_t *bci,
               const double *bcv, const int64_t *soff, int16_t *scol, double *sval,
               cudaStream_t s) {
  if (nblk > 0)
    k_sell_fill<<<(unsigned)nblk, kThreads, 0, s>>>(blk, nblk, brp, bci, bcv, soff, scol, sval);
}

void chunk_order(const int64_t *ptr, const CtaDesc *cta, int32_t ncta, int32_t *ord,
                 cudaStream_t s) {
  if (ncta > 0) k_chunk_order<<<(unsigned)ncta, kVecRows, 0, s>>>(ptr, cta, ord);
}

void sell_rows_width(const int64_t *ptr, const int64_t *srow0, const int32_t *srows,
                     int32_t nslice, const int32_t *rmap, int64_t *cnt, cudaStream_t s) {
  if (nslice > 0)
    k_sell_rows_width<<<grid_for(nslice, kThreads), kThreads, 0, s>>>(ptr, srow0, srows, nslice,
                                                                      rmap, cnt);
}

void sell_rows_fill(const int64_t *ptr, const int32_t *idx, const double *val,
                    const int64_t *srow0, const int32_t *srows, int32_t nslice,
                    const int32_t *rmap, const int64_t *off, int32_t *ocol, double *oval,
                    cudaStream_t s) {
  if (nslice > 0)
    k_sell_rows_fill<<<grid_for((int64_t)nslice * 32, kThreads), kThreads, 0, s>>>(
        ptr, idx, val, srow0, srows, nslice, rmap, off, ocol, oval);
}

void launch_gram_scatter(const BlockDesc *blk, const int32_t *blist, int32_t nlist,
                         const TileRow *trow, const int64_t *brp, const int32_t *bci,
                         const double *bcv, void *fac, int64_t fac_elems, int prec64,
                         cudaStream_t s) {
  if (nlist <= 0) return;
  // every tile of the listed blocks starts at zero (fac holds exactly their tiles)
  cudaMemsetAsync(fac, 0, (size_t)fac_elems * (prec64 ? sizeof(double) : sizeof(float)), s);
  if (prec64)
    k_gram_scatter<double><<<(unsigned)nlist, kThreads, 0, s>>>(
        blk, blist, trow, brp, bci, bcv, static_cast<double *>(fac));
  else
    k_gram_scatter<float><<<(unsigned)nlist, kThreads, 0, s>>>(
        blk, blist, trow, brp, bci, bcv, static_cast<float *>(fac));
}

}  // namespace cimmino
