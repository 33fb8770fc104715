// C ABI of the block Cimmino library (declared in include/cimmino.h).
//
// Setup pipeline (one launch per stage over all rows / blocks of all systems):
//   validate -> scale rows to unit 2-norm and permute (Sections 2.1-2.2) ->
//   transpose -> C = A A^T (Section 2.3) -> block-diagonal part G_i of C ->
//   tile envelope J0 -> scatter G_i into the tiled factor -> batched Cholesky ->
//   (FP32 mode) FP64 refactorisation of blocks with a poor pivot ratio.
// Solve: Algorithm 2 (Section 1.1) from x = 0, with every CG iteration a fixed
// sequence of five kernels, captured in a CUDA graph of check_every iterations;
// the host reads one status word per right-hand side between graph launches.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace cimmino;

namespace {

thread_local std::string g_last_error;

// Stream-ordered pool of device memory per device, owned by the library: freed blocks stay
// in the pool (release threshold: never) and serve the next context's allocations without a
// cudaMalloc, the way a framework's caching allocator does.
constexpr int kPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kPoolDevices] = {};

cudaMemPool_t library_pool() {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kPoolDevices) fail(CIMMINO_EUNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    CUDA_TRY(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = UINT64_MAX;
    CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}

// Device memory of one context or one standalone call: the caller's allocator when
// opts.alloc / opts.free are set, else the library pool, ordered on `stream`.
struct Allocator {
  cimmino_alloc_fn fa = nullptr;
  cimmino_free_fn ff = nullptr;
  void *user = nullptr;
  cudaStream_t stream = nullptr;

  void *get(size_t bytes) {
    void *p = nullptr;
    if (fa) {
      p = fa(bytes, stream, user);
      if (!p)
        fail(CIMMINO_ENOMEM, "the caller's allocator returned NULL for " +
                                 std::to_string(bytes) + " bytes");
      return p;
    }
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, library_pool(), stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(e == cudaErrorMemoryAllocation ? CIMMINO_ENOMEM : CIMMINO_ECUDA,
           "device allocation of " + std::to_string(bytes) + " bytes failed: " +
               cudaGetErrorString(e));
    }
    return p;
  }
  void put(void *p, size_t bytes) {
    if (!p) return;
    if (ff)
      ff(p, bytes, stream, user);
    else
      cudaFreeAsync(p, stream);
  }
};

// The allocator of the API call in progress on this host thread (set by AllocScope).
thread_local Allocator *t_alloc = nullptr;
struct AllocScope {
  Allocator *prev;
  explicit AllocScope(Allocator *a) : prev(t_alloc) { t_alloc = a; }
  ~AllocScope() { t_alloc = prev; }
  AllocScope(const AllocScope &) = delete;
  AllocScope &operator=(const AllocScope &) = delete;
};

// A device buffer from the allocator in scope at alloc() time, returned to the same
// allocator (which must outlive the buffer) on release.
template <typename T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  Allocator *a = nullptr;
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  ~DBuf() { release(); }
  void alloc(size_t count) {
    release();
    if (!t_alloc) fail(CIMMINO_ECUDA, "internal: device allocation outside an allocator scope");
    if (count == 0) count = 1;
    p = static_cast<T *>(t_alloc->get(count * sizeof(T)));
    a = t_alloc;
    n = count;
  }
  void release() {
    if (p) a->put(p, n * sizeof(T));
    p = nullptr;
    n = 0;
    a = nullptr;
  }
};

template <typename T>
void h2d(T *dst, const T *src, size_t count, cudaStream_t s) {
  if (count) CUDA_TRY(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyDefault, s));
}
template <typename T>
void d2h(T *dst, const T *src, size_t count, cudaStream_t s) {
  if (count) CUDA_TRY(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyDefault, s));
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  void start(cudaStream_t s) { cudaEventRecord(a, s); }
  double stop_ms(cudaStream_t s) {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
};

__global__ void k_interleave_to_cols(const double *__restrict__ x, int64_t N, int nrhs,
                                     double *__restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * nrhs) return;
  int64_t j = i / nrhs;
  int k = (int)(i % nrhs);
  out[(int64_t)k * N + j] = x[i];
}

__global__ void k_cols_to_interleaved(const double *__restrict__ v, int64_t N, int nrhs,
                                      double *__restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * nrhs) return;
  int64_t j = i / nrhs;
  int k = (int)(i % nrhs);
  out[i] = v[(int64_t)k * N + j];
}

}  // namespace

// The context's own stream, destroyed after every buffer of the context has been returned
// (members are destroyed in reverse order, so this one is declared first).
struct OwnedStream {
  cudaStream_t s = nullptr;
  ~OwnedStream() {
    if (s) cudaStreamDestroy(s);
  }
};

struct cimmino_ctx {
  OwnedStream owned;
  Allocator mem;  // declared before every DBuf member: outlives them
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cimmino_opts opts{};
  std::string err;
  int32_t nsys = 0;
  int64_t N = 0, nnz = 0;
  std::vector<SysDesc> hsys;
  std::vector<BlockDesc> hblk;
  std::vector<TileRow> htrow;
  std::vector<CtaDesc> hcta;
  int32_t max_mp = 0;
  int32_t proj_slots = 0, proj_slot_bytes = 0, proj_smem = 0, proj_wbytes = 8;
  int32_t proj_minb = 1;  // CTAs per SM of the projection kernel (autotuned with opts.tune)
  int32_t tuned = 0;      // 1: configuration measured here, 2: read from the tuning cache
  // matrices
  DBuf<int64_t> rp, cp, brp, crp;
  DBuf<int32_t> ci, ri, bci, cci, perm;
  DBuf<double> va, cv, d, bcv, ccv, rowabs, sval;
  DBuf<double> cs;  // column equilibration divisors (allocated when opts.ruiz_sweeps > 0)
  DBuf<int64_t> soff, aoff, toff;
  DBuf<int16_t> scol;
  DBuf<int32_t> acol, tcol;
  DBuf<int32_t> tord;  // A^T's rows in sliced-ELL position order (sorted inside CTA chunks)
  DBuf<double> aval, tval;
  DBuf<BlockDesc> blk;
  DBuf<int32_t> border;  // projection launch order (longest first)
  std::vector<int32_t> hborder;
  DBuf<int32_t> mr_list;  // multi-RHS launch order: tensor-core blocks first
  int32_t mr_ntc = 0;     // blocks the tensor-core multi-RHS kernel takes
  std::vector<unsigned char> tmaps;  // its 4 tensor maps (host copies, passed by value)
  DBuf<TileRow> trow;
  DBuf<SysDesc> sys;
  DBuf<CtaDesc> cta;
  DBuf<float> fac32, dinv32, facT32, dinvT32, dinvP32, dinvTP32;
  DBuf<double> fac64, dinv64, facT64, dinvT64, dinvP64, dinvTP64;
  DBuf<TileRow> trowT;
  std::vector<TileRow> htrowT;
  int64_t pass_bytes = 0;  // factor bytes one forward + backward solve pass streams
  int64_t nnzc = 0, nnz_bd = 0, factor_bytes = 0;
  double factor_flops = 0.0;  // algorithmic flops of the envelope Cholesky of all G_i
  double t_chol_ms = 0.0;     // device time of the batched Cholesky launch alone
  int32_t fallbacks = 0;
  int32_t chol_split = 0;  // FP64 Cholesky blocks shared by two CTAs
  int64_t setup_launches = 0;  // kernels launched by the setup
  double t_setup_ms = 0.0, t_factor_ms = 0.0;
  bool have_aat = false;
  // solve state
  int32_t nrhs = 0;
  DBuf<LaneState> lane;
  DBuf<double> fs, x, p, r, psi, u, y, part, Fin, stats4;
  DBuf<int32_t> cnt, refine_max, err_flag;
  DBuf<int64_t> refine_total;
  cudaGraphExec_t graph = nullptr;
  int32_t graph_nrhs = 0, graph_iters = 0;
  IterArgs args{};
  // opts.time_proj: events around the projection launches of one check interval, and the
  // live projection time of the last solve
  std::vector<cudaEvent_t> pev;
  double proj_ms_total = 0.0;
  int64_t proj_launches = -1;

  ~cimmino_ctx() {
    if (graph) cudaGraphExecDestroy(graph);
    for (cudaEvent_t e : pev) cudaEventDestroy(e);
  }
};

namespace {

void opts_default(cimmino_opts *o) {
  std::memset(o, 0, sizeof(*o));
  o->precision = CIMMINO_FP64;
  o->layout = CIMMINO_LAYOUT_SKYLINE;
  o->tile = 0;
  o->refine_max = 6;
  o->refine_tol = 1e-12;
  o->pivot_ratio_min = 1e-4;
  o->max_iter = 10000;
  o->use_graph = 1;
  o->check_every = 8;
  o->keep_aat = 0;
  o->multi_rhs = 1;
  o->refine_relax = 0;
  o->ruiz_sweeps = 0;
  o->time_proj = 0;
  o->stream = nullptr;
  o->alloc = nullptr;
  o->free = nullptr;
  o->alloc_user = nullptr;
  o->tune = 0;
  o->tune_cache = nullptr;
}

void check_opts(const cimmino_opts &o) {
  if (o.precision != CIMMINO_FP64 && o.precision != CIMMINO_FP32_REFINE)
    fail(CIMMINO_EINVAL, "opts.precision must be CIMMINO_FP64 or CIMMINO_FP32_REFINE");
  if (o.layout != CIMMINO_LAYOUT_DENSE && o.layout != CIMMINO_LAYOUT_SKYLINE)
    fail(CIMMINO_EINVAL, "opts.layout must be CIMMINO_LAYOUT_DENSE or CIMMINO_LAYOUT_SKYLINE");
  if (o.tile != 0 && o.tile != kTile) fail(CIMMINO_EUNSUPPORTED, "opts.tile must be 0 or 64");
  if (o.refine_max < 0 || o.refine_max > 64) fail(CIMMINO_EINVAL, "opts.refine_max not in [0,64]");
  if (!(o.refine_tol >= 0.0)) fail(CIMMINO_EINVAL, "opts.refine_tol must be >= 0");
  if (o.max_iter < 0) fail(CIMMINO_EINVAL, "opts.max_iter must be >= 0");
  if (o.check_every < 1 || o.check_every > 1024)
    fail(CIMMINO_EINVAL, "opts.check_every not in [1,1024]");
  if (o.ruiz_sweeps < 0 || o.ruiz_sweeps > 100)
    fail(CIMMINO_EINVAL, "opts.ruiz_sweeps not in [0,100]");
  if (o.time_proj != 0 && o.time_proj != 1) fail(CIMMINO_EINVAL, "opts.time_proj must be 0 or 1");
  if ((o.alloc == nullptr) != (o.free == nullptr))
    fail(CIMMINO_EINVAL, "opts.alloc and opts.free must be set together");
  if (o.tune != 0 && o.tune != 1) fail(CIMMINO_EINVAL, "opts.tune must be 0 or 1");
  if (o.multi_rhs < 0 || o.multi_rhs > 2) fail(CIMMINO_EINVAL, "opts.multi_rhs not in [0,2]");
}

// One NVTX range per stage (header-only NVTX 3: a no-op unless a profiler attaches), so
// that a trace, or an ncu capture filtered with --nvtx, can select a stage.
class Stages {
 public:
  explicit Stages(const char *first) { nvtxRangePushA(first); }
  void next(const char *name) {
    nvtxRangePop();
    nvtxRangePushA(name);
  }
  ~Stages() { nvtxRangePop(); }
  Stages(const Stages &) = delete;
  Stages &operator=(const Stages &) = delete;
};

// ------------------------------------------------------------------ setup
// ---- static schedule of the FP64 Cholesky (k_cholesky)
// Cost of a block in units of one full trailing-update tile of k_cholesky (81 us on GB300),
// with weights fitted to the measured times of the 512 blocks of the n = 2^20 random workload
// (1.9% mean error): a diagonal tile's factor and inverse 1.41 (a serial pivot chain, partly
// hidden by the look-ahead), a solved tile (I, K) with the symmetric update of (I, I) 0.59.
constexpr double kCostDiag = 1.41, kCostTrsmSym = 0.59;
// A pair barrier of a split block (a few L2 round trips), in the same unit.
constexpr double kCostPairSync = 0.03;
// A block whose cost reaches this fraction of the mean load per CTA is split over two CTAs.
constexpr double kSplitFraction = 0.9;

struct CholPlan {
  std::vector<CholItem> items;
  std::vector<int32_t> ptr;  // ncta + 1
  int32_t nsplit = 0;
  double makespan = 0.0;  // largest list, in cost units
};

// Cost of one block from its tile counts: nt diagonal tiles, ntrsm solved tiles (I, K) (each
// with the symmetric update of (I, I)) and nfull full trailing updates; diag: the part of it
// on the diagonal tiles, sync: the pair barriers of one half when the block is split.
void chol_block_cost(int32_t nt, int64_t ntrsm, int64_t nfull, double &cost, double &diag,
                     double &sync) {
  diag = kCostDiag * nt;
  cost = diag + kCostTrsmSym * (double)ntrsm + (double)nfull;
  sync = 3.0 * kCostPairSync * nt;
}

// First-fit decreasing of jobs (sorted by decreasing cost) into bins of capacity cap on top of
// the loads `load`; false if a job fits nowhere.
bool ffd_pack(const std::vector<int32_t> &jobs, const std::vector<double> &cost, double cap,
              std::vector<double> load, std::vector<int32_t> &bin_of) {
  for (size_t q = 0; q < jobs.size(); ++q) {
    const double w = cost[jobs[q]];
    size_t k = 0;
    while (k < load.size() && load[k] + w > cap) ++k;
    if (k == load.size()) return false;
    load[k] += w;
    bin_of[q] = (int32_t)k;
  }
  return true;
}

// Schedule with the ns largest blocks split: their halves (the diagonal part plus half of the
// rest, plus three pair barriers per tile column) first in CTAs 2i and 2i+1, the other blocks
// packed by MULTIFIT: the smallest capacity that first-fit decreasing fills, found by bisection
// between the lower bound and the greedy longest-first makespan.  Returns the makespan.
double pack_cholesky(const std::vector<int32_t> &order, const std::vector<double> &cost,
                     const std::vector<double> &diag, const std::vector<double> &sync,
                     int32_t maxcta, int32_t ns, CholPlan &P) {
  const int32_t n = (int32_t)order.size();
  const int32_t ncta = std::min(maxcta, n + ns);
  std::vector<double> load(ncta, 0.0);
  for (int32_t i = 0; i < ns; ++i) {
    const int32_t b = order[i];
    load[2 * i] = load[2 * i + 1] = diag[b] + 0.5 * (cost[b] - diag[b]) + sync[b];
  }
  std::vector<int32_t> jobs(order.begin() + ns, order.end());
  std::vector<int32_t> bin_of(jobs.size(), 0);
  // greedy longest-first (list scheduling): a feasible capacity
  std::vector<double> l(load);
  for (size_t q = 0; q < jobs.size(); ++q) {
    const size_t k = (size_t)(std::min_element(l.begin(), l.end()) - l.begin());
    l[k] += cost[jobs[q]];
    bin_of[q] = (int32_t)k;
  }
  double hi = 0.0, sum = 0.0, big = 0.0;
  for (double x : l) hi = std::max(hi, x);
  for (double x : load) sum += x, big = std::max(big, x);
  for (int32_t b : jobs) sum += cost[b], big = std::max(big, cost[b]);
  double lo = std::max(big, sum / ncta);
  std::vector<int32_t> trial(jobs.size());
  for (int it = 0; it < 32 && hi - lo > 1e-6 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (ffd_pack(jobs, cost, mid, load, trial)) {
      hi = mid;
      bin_of = trial;
    } else {
      lo = mid;
    }
  }
  // local search: move a job out of the most loaded CTA, or swap it for a smaller one, while
  // that lowers the maximum (bounded number of rounds; long lists are packed finely enough)
  std::vector<double> bl(load);
  for (size_t q = 0; q < jobs.size(); ++q) bl[bin_of[q]] += cost[jobs[q]];
  const int rounds = jobs.size() <= 4096 ? 4 * ncta : 0;
  for (int round = 0; round < rounds; ++round) {
    const int32_t h = (int32_t)(std::max_element(bl.begin(), bl.end()) - bl.begin());
    double best = 1e-9 * bl[h];
    size_t bq = 0, bi = 0;
    int32_t bk = -1;
    bool swap = false;
    for (size_t q = 0; q < jobs.size(); ++q) {
      if (bin_of[q] != h) continue;
      const double cq = cost[jobs[q]];
      for (size_t i = 0; i < jobs.size(); ++i) {  // swaps (q <-> i), i in another CTA
        const int32_t k = bin_of[i];
        const double d = cq - cost[jobs[i]];
        if (k == h || d <= 0.0 || bl[k] + d >= bl[h]) continue;
        const double gain = bl[h] - std::max(bl[h] - d, bl[k] + d);
        if (gain > best) best = gain, bq = q, bi = i, bk = k, swap = true;
      }
      for (int32_t k = 0; k < ncta; ++k) {  // moves
        if (k == h || bl[k] + cq >= bl[h]) continue;
        const double gain = bl[h] - std::max(bl[h] - cq, bl[k] + cq);
        if (gain > best) best = gain, bq = q, bk = k, swap = false;
      }
    }
    if (bk < 0) break;
    bl[h] -= cost[jobs[bq]];
    bl[bk] += cost[jobs[bq]];
    bin_of[bq] = bk;
    if (swap) {
      bl[bk] -= cost[jobs[bi]];
      bl[h] += cost[jobs[bi]];
      bin_of[bi] = h;
    }
  }
  std::vector<std::vector<CholItem>> lists(ncta);
  for (int32_t i = 0; i < ns; ++i) {
    lists[2 * i].push_back(CholItem{order[i], 0, 2, i});
    lists[2 * i + 1].push_back(CholItem{order[i], 1, 2, i});
  }
  for (size_t q = 0; q < jobs.size(); ++q) lists[bin_of[q]].push_back(CholItem{jobs[q], 0, 1, 0});
  P.items.clear();
  P.ptr.assign(1, 0);
  double makespan = 0.0;
  for (int32_t k = 0; k < ncta; ++k) {
    double t = load[k];  // the split half, if any
    for (const CholItem &it : lists[k]) {
      P.items.push_back(it);
      if (it.nparts == 1) t += cost[it.b];
    }
    P.ptr.push_back((int32_t)P.items.size());
    makespan = std::max(makespan, t);
  }
  P.nsplit = ns;
  P.makespan = makespan;
  return makespan;
}

// blocks: the blocks to factor; cost / diag: their costs and the diagonal-tile part of them;
// nt: their tile rows; maxcta: CTAs that can be resident at once.  Tries a ladder of split
// counts among the blocks whose cost reaches kSplitFraction of the mean load per CTA and keeps
// the smallest count with the shortest makespan.
CholPlan plan_cholesky(const std::vector<int32_t> &blocks, const std::vector<double> &cost,
                       const std::vector<double> &diag, const std::vector<double> &sync,
                       int32_t maxcta, bool allow_split) {
  CholPlan best;
  std::vector<int32_t> order(blocks);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
  const int32_t n = (int32_t)order.size();
  if (n == 0 || maxcta <= 0) {
    best.ptr.assign(1, 0);
    return best;
  }
  double total = 0.0;
  for (int32_t b : order) total += cost[b];
  int32_t nmax = 0;
  while (allow_split && nmax < n && 2 * (nmax + 1) <= maxcta &&
         cost[order[nmax]] >= kSplitFraction * total / maxcta)
    ++nmax;
  std::vector<int32_t> ladder;
  for (int32_t ns = 1; ns < nmax; ns = ns < 4 ? ns + 1 : ns + ns / 2) ladder.push_back(ns);
  if (nmax > 0) ladder.push_back(nmax);
  double best_t = pack_cholesky(order, cost, diag, sync, maxcta, 0, best);
  for (int32_t ns : ladder) {
    CholPlan P;
    const double t = pack_cholesky(order, cost, diag, sync, maxcta, ns, P);
    if (t < best_t * (1.0 - 1e-3)) {
      best_t = t;
      best = std::move(P);
    }
  }
  return best;
}

// Uploads a plan and runs k_cholesky on it (the flags and the error word zeroed first);
// returns after the launch, the buffers stay alive in `keep` until the caller synchronises.
// A plan with split blocks needs all its CTAs resident at once (a cooperative launch); if the
// device refuses that (other work holding SMs), `replan` (the same blocks without splits) runs
// as a plain grid instead.  Returns the split blocks of the plan that ran.
struct CholLaunchBufs {
  DBuf<CholItem> items;
  DBuf<int32_t> ptr, flags, err;
};
template <typename Replan>
int32_t run_cholesky64(cimmino_ctx *c, const CholPlan &P, Replan replan, double *pmin,
                       int32_t *pfail, CholLaunchBufs &keep, cudaStream_t s) {
  auto run = [&](const CholPlan &Q) {
    const int32_t ncta = (int32_t)Q.ptr.size() - 1;
    keep.items.alloc(Q.items.size());
    keep.ptr.alloc(Q.ptr.size());
    keep.flags.alloc(std::max<int32_t>(2 * Q.nsplit, 1));
    keep.err.alloc(1);
    h2d(keep.items.p, Q.items.data(), Q.items.size(), s);
    h2d(keep.ptr.p, Q.ptr.data(), Q.ptr.size(), s);
    CUDA_TRY(cudaMemsetAsync(keep.flags.p, 0, keep.flags.n * sizeof(int32_t), s));
    CUDA_TRY(cudaMemsetAsync(keep.err.p, 0, sizeof(int32_t), s));
    return launch_cholesky(c->blk.p, keep.items.p, keep.ptr.p, ncta, Q.nsplit > 0, c->trow.p,
                           c->fac64.p, c->dinv64.p, pmin, pfail, keep.flags.p, keep.err.p, s);
  };
  if ((int32_t)P.ptr.size() - 1 <= 0) return 0;
  cudaError_t e = run(P);
  if (P.nsplit > 0 && e == cudaErrorCooperativeLaunchTooLarge) {
    (void)cudaGetLastError();  // a refused launch ran nothing
    const CholPlan Q = replan();
    CUDA_TRY(run(Q));
    return Q.nsplit;
  }
  CUDA_TRY(e);
  return P.nsplit;
}

// Resident CTAs of k_cholesky and whether a schedule may split blocks (cooperative launch).
void cholesky_capacity(int32_t &maxcta, bool &allow_split) {
  int dev = 0, coop = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  maxcta = cholesky_resident_ctas();
  if (maxcta <= 0) fail(CIMMINO_ECUDA, "k_cholesky cannot be resident on this device");
  allow_split = coop != 0;
}

void setup_impl(cimmino_ctx *c, int32_t nsys, const cimmino_csr *A, const int32_t *K,
                const int32_t *const *perms, const int64_t *const *bps) {
  cudaStream_t s = c->stream;
  c->nsys = nsys;
  Stages stage("cimmino.setup.validate");
  // ---- host-side validation and global layout
  int64_t N = 0, NNZ = 0;
  c->hsys.resize(nsys);
  for (int32_t q = 0; q < nsys; ++q) {
    const cimmino_csr &M = A[q];
    if (M.n <= 0 || M.nnz < 0 || !M.row_ptr || !M.col_idx || (M.nnz > 0 && !M.val))
      fail(CIMMINO_EINVAL, "system " + std::to_string(q) + ": bad CSR header");
    if (K[q] < 1 || K[q] > M.n) fail(CIMMINO_EINVAL, "K must be in [1, n]");
    if (!bps || !bps[q]) fail(CIMMINO_EINVAL, "block_ptr is NULL");
    const int64_t *bp = bps[q];
    if (bp[0] != 0 || bp[K[q]] != M.n) fail(CIMMINO_EINVAL, "block_ptr must start at 0 and end at n");
    for (int32_t b = 0; b < K[q]; ++b) {
      if (bp[b + 1] <= bp[b]) fail(CIMMINO_EINVAL, "block_ptr must be strictly increasing");
      if (bp[b + 1] - bp[b] > kMaxBlockRows)
        fail(CIMMINO_EUNSUPPORTED, "a block has more than 4096 rows");
    }
    const int32_t *pm = perms ? perms[q] : nullptr;
    if (pm && nsys > 1) {  // one system: checked on the device below
      std::vector<char> seen(M.n, 0);
      for (int64_t r = 0; r < M.n; ++r) {
        if (pm[r] < 0 || pm[r] >= M.n || seen[pm[r]])
          fail(CIMMINO_EINVAL, "perm is not a permutation of 0..n-1");
        seen[pm[r]] = 1;
      }
    }
    c->hsys[q].row0 = N;
    c->hsys[q].n = M.n;
    N += M.n;
    NNZ += M.nnz;
  }
  if (N >= (int64_t(1) << 31) - 1) fail(CIMMINO_EUNSUPPORTED, "total rows exceed 2^31 - 1");
  c->N = N;
  c->nnz = NNZ;

  Timer tsetup;
  tsetup.start(s);
  // ---- concatenated unscaled matrix A0 (block-diagonal over systems)
  DBuf<int64_t> rp0;
  DBuf<int32_t> ci0;
  DBuf<double> v0;
  const int64_t *drp0;
  const int32_t *dci0;
  const double *dv0;
  if (nsys == 1 && A[0].on_device) {
    drp0 = A[0].row_ptr;
    dci0 = A[0].col_idx;
    dv0 = A[0].val;
  } else if (nsys == 1) {
    rp0.alloc(N + 1);
    ci0.alloc(NNZ);
    v0.alloc(NNZ);
    h2d(rp0.p, A[0].row_ptr, N + 1, s);
    h2d(ci0.p, A[0].col_idx, NNZ, s);
    h2d(v0.p, A[0].val, NNZ, s);
    drp0 = rp0.p;
    dci0 = ci0.p;
    dv0 = v0.p;
  } else {
    std::vector<int64_t> hrp(N + 1);
    std::vector<int32_t> hci(NNZ);
    std::vector<double> hv(NNZ);
    int64_t z = 0;
    for (int32_t q = 0; q < nsys; ++q) {
      const cimmino_csr &M = A[q];
      std::vector<int64_t> trp(M.n + 1);
      const int64_t *srp = M.row_ptr;
      const int32_t *sci = M.col_idx;
      const double *sv = M.val;
      std::vector<int32_t> tci;
      std::vector<double> tv;
      if (M.on_device) {
        CUDA_TRY(cudaMemcpy(trp.data(), M.row_ptr, sizeof(int64_t) * (M.n + 1), cudaMemcpyDefault));
        tci.resize(M.nnz);
        tv.resize(M.nnz);
        CUDA_TRY(cudaMemcpy(tci.data(), M.col_idx, sizeof(int32_t) * M.nnz, cudaMemcpyDefault));
        CUDA_TRY(cudaMemcpy(tv.data(), M.val, sizeof(double) * M.nnz, cudaMemcpyDefault));
        srp = trp.data();
        sci = tci.data();
        sv = tv.data();
      }
      if (srp[0] != 0 || srp[M.n] != M.nnz)
        fail(CIMMINO_EINVAL, "system " + std::to_string(q) + ": row_ptr ends do not match nnz");
      const int64_t r0 = c->hsys[q].row0;
      for (int64_t i = 0; i < M.n; ++i) hrp[r0 + i] = z + srp[i];
      for (int64_t e = 0; e < M.nnz; ++e) {
        hci[z + e] = sci[e] < 0 || sci[e] >= M.n ? -1 : (int32_t)(sci[e] + r0);
        hv[z + e] = sv[e];
      }
      z += M.nnz;
    }
    hrp[N] = z;
    rp0.alloc(N + 1);
    ci0.alloc(NNZ);
    v0.alloc(NNZ);
    h2d(rp0.p, hrp.data(), N + 1, s);
    h2d(ci0.p, hci.data(), NNZ, s);
    h2d(v0.p, hv.data(), NNZ, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    drp0 = rp0.p;
    dci0 = ci0.p;
    dv0 = v0.p;
  }
  DBuf<int32_t> flag;
  flag.alloc(4);
  CUDA_TRY(cudaMemsetAsync(flag.p, 0, 4 * sizeof(int32_t), s));
  launch_validate_csr(drp0, dci0, N, NNZ, flag.p, s);
  c->setup_launches += 1;
  // the row permutation (concatenated systems: each system's rows map into its own range);
  // a single system's is copied as given and checked on the device (flag[3])
  c->perm.alloc(N);
  if (nsys == 1 && perms && perms[0]) {
    h2d(c->perm.p, perms[0], N, s);
    DBuf<int32_t> seen;
    seen.alloc(N);
    CUDA_TRY(cudaMemsetAsync(seen.p, 0, sizeof(int32_t) * N, s));
    launch_check_perm(c->perm.p, N, seen.p, flag.p + 3, s);
    c->setup_launches += 1;
  } else {
    std::vector<int32_t> hperm(N);
    for (int32_t q = 0; q < nsys; ++q) {
      const int64_t r0 = c->hsys[q].row0;
      const int32_t *pm = perms ? perms[q] : nullptr;
      for (int64_t r = 0; r < c->hsys[q].n; ++r) hperm[r0 + r] = (int32_t)(r0 + (pm ? pm[r] : r));
    }
    h2d(c->perm.p, hperm.data(), N, s);
  }
  int32_t hflag[4] = {0, 0, 0, 0};
  d2h(hflag, flag.p, 4, s);
  CUDA_TRY(cudaStreamSynchronize(s));
  if (hflag[0]) {
    std::string why = (hflag[0] & 1) ? "row_ptr not monotone or inconsistent with nnz"
                      : (hflag[0] & 2) ? "column index out of range"
                                       : "column indices not strictly increasing within a row";
    fail(CIMMINO_EINVAL, "malformed CSR: " + why);
  }
  if (hflag[3]) fail(CIMMINO_EINVAL, "perm is not a permutation of 0..n-1");
  stage.next("cimmino.setup.scale");
  // ---- row and column equilibration (Section 3.1), in place on our own copy of A's values
  DBuf<double> rs;
  if (c->opts.ruiz_sweeps > 0) {
    if (dv0 != v0.p) {  // caller-owned device values: copy before scaling
      v0.alloc(NNZ);
      CUDA_TRY(cudaMemcpyAsync(v0.p, dv0, sizeof(double) * NNZ, cudaMemcpyDefault, s));
      dv0 = v0.p;
    }
    DBuf<double> work;
    work.alloc(3 * N);
    rs.alloc(N);
    c->cs.alloc(N);
    launch_equilibrate(drp0, dci0, v0.p, N, c->opts.ruiz_sweeps, rs.p, c->cs.p, work.p, s);
    c->setup_launches += 1 + 3 * c->opts.ruiz_sweeps;
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  // ---- blocks
  int32_t ntrow = 0, nslice = 0;
  c->max_mp = 0;
  for (int32_t q = 0; q < nsys; ++q) {
    for (int32_t b = 0; b < K[q]; ++b) {
      BlockDesc B{};
      B.row0 = c->hsys[q].row0 + bps[q][b];
      B.m = (int32_t)(bps[q][b + 1] - bps[q][b]);
      B.nt = (B.m + kTile - 1) / kTile;
      B.trow0 = ntrow;
      B.sys = q;
      B.prec64 = c->opts.precision == CIMMINO_FP64;
      B.slice0 = nslice;
      nslice += (B.m + 31) / 32;
      ntrow += B.nt;
      c->max_mp = std::max(c->max_mp, B.nt * kTile);
      c->hblk.push_back(B);
    }
  }
  const int32_t nblk = (int32_t)c->hblk.size();
  c->blk.alloc(nblk);
  h2d(c->blk.p, c->hblk.data(), nblk, s);
  if (proj_smem_bytes(c->max_mp, 2, kTile * kTile * 8, 8) > kProjSmemMax)
    fail(CIMMINO_EUNSUPPORTED, "block too large for the projection kernel");

  // ---- scale and permute rows (Sections 2.1, 2.2)
  DBuf<int64_t> len, tmp;
  const int64_t tl = scan_tmp_len(N);
  len.alloc(2 * N);
  tmp.alloc(tl);
  c->rp.alloc(N + 1);
  launch_permuted_lengths(drp0, c->perm.p, N, len.p, s);
  launch_scan_counts(len.p, c->rp.p, N, tmp.p, tl, s);
  c->setup_launches += 4;  // lengths + 3-pass scan
  c->ci.alloc(NNZ);
  c->va.alloc(NNZ);
  c->d.alloc(N);
  launch_scale_permute(drp0, dci0, dv0, c->perm.p, c->rp.p, N, c->ci.p, c->va.p, c->d.p,
                       c->opts.ruiz_sweeps > 0 ? rs.p : nullptr, flag.p + 1, s);
  c->setup_launches += 1;
  // ---- transpose
  c->cp.alloc(N + 1);
  c->ri.alloc(NNZ);
  c->cv.alloc(NNZ);
  launch_transpose(c->rp.p, c->ci.p, c->va.p, N, NNZ, c->cp.p, c->ri.p, c->cv.p, len.p, tmp.p,
                   tl, s);
  c->setup_launches += 6;  // count, 3-pass scan, fill, sort
  d2h(hflag + 1, flag.p + 1, 1, s);
  CUDA_TRY(cudaStreamSynchronize(s));
  if (hflag[1]) fail(CIMMINO_ESINGULAR, "A has a zero row (the matrix is singular)");
  rp0.release();
  ci0.release();
  v0.release();
  rs.release();

  stage.next("cimmino.setup.aat");
  // ---- C = A A^T (Section 2.3).  The solve needs only its block-diagonal part, the Gram
  // blocks G_i: unless the caller keeps C (opts.keep_aat), every row gathers only the
  // candidates of its own block (a window of each sorted column of the transpose), and the
  // SpGEMM writes G_i directly.  Its values are those entries of C, bit for bit.
  DBuf<int64_t> cntc;
  DBuf<int32_t> ovf;
  DBuf<int32_t> rowblk, rowmin;
  cntc.alloc(N);
  ovf.alloc(N + 1);
  rowblk.alloc(N);
  rowmin.alloc(N);
  launch_row_block_ids(c->blk.p, nblk, rowblk.p, s);
  const bool full_c = c->opts.keep_aat != 0;
  const BlockDesc *wblk = full_c ? nullptr : c->blk.p;
  const int32_t *wrow = full_c ? nullptr : rowblk.p;
  spgemm_count(c->rp.p, c->ci.p, c->cp.p, c->ri.p, N, cntc.p, ovf.p + 1, ovf.p, s, wblk, wrow);
  c->setup_launches += 2;
  int32_t novf = 0;
  d2h(&novf, ovf.p, 1, s);
  CUDA_TRY(cudaStreamSynchronize(s));
  if (novf > 0) {
    spgemm_overflow(c->rp.p, c->ci.p, c->va.p, c->cp.p, c->ri.p, ovf.p + 1, novf, cntc.p, nullptr,
                    nullptr, nullptr, flag.p + 2, s, wblk, wrow);
    d2h(hflag + 2, flag.p + 2, 1, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hflag[2])
      fail(CIMMINO_EUNSUPPORTED, "a row of A A^T has more than 8192 structural candidates");
  }
  DBuf<int64_t> &orp = full_c ? c->crp : c->brp;
  orp.alloc(N + 1);
  launch_scan_counts(cntc.p, orp.p, N, tmp.p, tl, s);
  c->setup_launches += 3 + (novf > 0 ? 2 : 0);
  int64_t nout = 0;
  d2h(&nout, orp.p + N, 1, s);
  CUDA_TRY(cudaStreamSynchronize(s));
  DBuf<int32_t> &oci = full_c ? c->cci : c->bci;
  DBuf<double> &ocv = full_c ? c->ccv : c->bcv;
  oci.alloc(nout);
  ocv.alloc(nout);
  spgemm_fill(c->rp.p, c->ci.p, c->va.p, c->cp.p, c->ri.p, c->cv.p, N, orp.p, oci.p, ocv.p, s,
              wblk, wrow);
  c->setup_launches += 1;
  if (novf > 0)
    spgemm_overflow(c->rp.p, c->ci.p, c->va.p, c->cp.p, c->ri.p, ovf.p + 1, novf, cntc.p, orp.p,
                    oci.p, ocv.p, flag.p + 2, s, wblk, wrow);

  // ---- block-diagonal part of C: the Gram blocks G_i (exact, FP64, local columns)
  if (full_c) {
    c->nnzc = nout;
    c->have_aat = true;
    bd_count(c->crp.p, c->cci.p, c->blk.p, rowblk.p, N, cntc.p, s);
    c->brp.alloc(N + 1);
    launch_scan_counts(cntc.p, c->brp.p, N, tmp.p, tl, s);
    c->setup_launches += 4;  // count, 3-pass scan
    d2h(&c->nnz_bd, c->brp.p + N, 1, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    c->bci.alloc(c->nnz_bd);
    c->bcv.alloc(c->nnz_bd);
    bd_fill(c->crp.p, c->cci.p, c->ccv.p, c->blk.p, rowblk.p, N, c->brp.p, c->bci.p, c->bcv.p,
            rowmin.p, s);
  } else {
    c->nnzc = 0;
    c->nnz_bd = nout;
    bd_localize(c->brp.p, c->bci.p, c->blk.p, rowblk.p, N, rowmin.p, s);
  }
  c->setup_launches += 2;  // fill or local columns, tile envelope
  // sliced-ELL copy of the Gram blocks for the refinement residual
  {
    DBuf<int64_t> scnt;
    scnt.alloc(nslice);
    c->soff.alloc(nslice + 1);
    sell_width(c->blk.p, nblk, c->brp.p, scnt.p, s);
    launch_scan_counts(scnt.p, c->soff.p, nslice, tmp.p, tl, s);
    int64_t sn = 0;
    d2h(&sn, c->soff.p + nslice, 1, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    c->scol.alloc(sn);
    c->sval.alloc(sn);
    sell_fill(c->blk.p, nblk, c->brp.p, c->bci.p, c->bcv.p, c->soff.p, c->scol.p, c->sval.p, s);
    c->setup_launches += 5;  // widths, 3-pass scan, fill
  }

  // ---- tile envelope and factor layout
  DBuf<int32_t> dj0;
  dj0.alloc(ntrow);
  launch_tile_j0(c->blk.p, nblk, rowmin.p, c->opts.layout == CIMMINO_LAYOUT_DENSE, dj0.p, s);
  std::vector<int32_t> hj0(ntrow);
  d2h(hj0.data(), dj0.p, ntrow, s);
  CUDA_TRY(cudaStreamSynchronize(s));
  c->htrow.resize(ntrow);
  int64_t off = 0, doff = 0;
  const int64_t TT = (int64_t)kTile * kTile;
  for (auto &B : c->hblk) {
    B.dinv_off = doff;
    doff += (int64_t)B.nt * TT;
    for (int32_t I = 0; I < B.nt; ++I) {
      TileRow &R = c->htrow[B.trow0 + I];
      R.j0 = hj0[B.trow0 + I];
      R.off = off;
      off += (int64_t)(I - R.j0 + 1) * TT;
    }
  }
  c->trow.alloc(ntrow);
  h2d(c->trow.p, c->htrow.data(), ntrow, s);
  h2d(c->blk.p, c->hblk.data(), nblk, s);
  const bool fp64 = c->opts.precision == CIMMINO_FP64;
  if (fp64) {
    c->fac64.alloc(off);
    c->dinv64.alloc(doff);
  } else {
    c->fac32.alloc(off);
    c->dinv32.alloc(doff);
  }
  c->factor_bytes = off * (fp64 ? 8 : 4);
  // Algorithmic flops of the Cholesky restricted to the tile envelope, with the actual rows
  // r_I of every tile row: the diagonal factorisations r_K^3 / 3, the triangular solves
  // r_I r_K^2 of the tiles (I, K) below them, and the trailing products 2 r_I r_J r_K
  // (r_I^2 r_K on the symmetric diagonal tiles J = I) for K < J <= I inside the envelope.
  // Also the cost of every block for the FP64 Cholesky's schedule (tile counts weighted
  // with the per-phase times of k_cholesky).
  c->factor_flops = 0.0;
  std::vector<double> blk_flops(nblk, 0.0), chol_cost(nblk, 0.0), chol_diag(nblk, 0.0),
      chol_sync(nblk, 0.0);
  for (int32_t b = 0; b < nblk; ++b) {
    const BlockDesc &B = c->hblk[b];
    auto rows = [&](int32_t I) { return (double)std::min(kTile, B.m - I * kTile); };
    double f = 0.0;
    int64_t ntrsm = 0, nfull = 0;
    for (int32_t K = 0; K < B.nt; ++K) {
      const double rK = rows(K);
      f += rK * rK * rK / 3.0;
      for (int32_t I = K + 1; I < B.nt; ++I) {
        if (c->htrow[B.trow0 + I].j0 > K) continue;
        const double rI = rows(I);
        f += rI * rK * rK + rI * rI * rK;  // solve of (I, K), update of (I, I)
        ++ntrsm;
        for (int32_t J = K + 1; J < I; ++J)
          if (c->htrow[B.trow0 + J].j0 <= K) {
            f += 2.0 * rI * rows(J) * rK;
            ++nfull;
          }
      }
    }
    blk_flops[b] = f;
    c->factor_flops += f;
    chol_block_cost(B.nt, ntrsm, nfull, chol_cost[b], chol_diag[b], chol_sync[b]);
  }
  c->t_setup_ms = tsetup.stop_ms(s);

  stage.next("cimmino.setup.factor");
  // ---- batched Cholesky of all G_i
  Timer tfac;
  tfac.start(s);
  // one CTA per block, launched in order of decreasing work (longest first): the blocks
  // that take longest start in the first wave and the short ones fill in behind them
  std::vector<int32_t> hlist(nblk);
  for (int32_t b = 0; b < nblk; ++b) hlist[b] = b;
  std::stable_sort(hlist.begin(), hlist.end(),
                   [&](int32_t x, int32_t y) { return blk_flops[x] > blk_flops[y]; });
  DBuf<int32_t> blist, pfail;
  DBuf<double> pmin;
  blist.alloc(nblk);
  pfail.alloc(nblk);
  pmin.alloc(nblk);
  h2d(blist.p, hlist.data(), nblk, s);
  void *fac = fp64 ? (void *)c->fac64.p : (void *)c->fac32.p;
  launch_gram_scatter(c->blk.p, blist.p, nblk, c->trow.p, c->brp.p, c->bci.p, c->bcv.p, fac,
                      fp64 ? (int64_t)c->fac64.n : (int64_t)c->fac32.n, fp64, s);
  if (!fp64) {
    c->err_flag.alloc(1);
    CUDA_TRY(cudaMemsetAsync(c->err_flag.p, 0, sizeof(int32_t), s));
  }
  DBuf<float> tc_scratch;  // the split operand copy of L (FP32 blocks), freed after setup
  DBuf<int32_t> tc_rowblk;
  if (!fp64) {
    tc_scratch.alloc(cholesky_tc_scratch_floats(off));
    tc_rowblk.alloc(ntrow);
  }
  // FP64: a static schedule over the resident CTAs (built before the timer starts)
  CholPlan plan;
  CholLaunchBufs cbufs;
  int32_t maxcta = 0;
  bool allow_split = false;
  if (fp64) {
    cholesky_capacity(maxcta, allow_split);
    plan = plan_cholesky(hlist, chol_cost, chol_diag, chol_sync, maxcta, allow_split);
  }
  Timer tchol;
  tchol.start(s);
  if (fp64) {
    c->chol_split = run_cholesky64(
        c, plan,
        [&] { return plan_cholesky(hlist, chol_cost, chol_diag, chol_sync, maxcta, false); },
        pmin.p, pfail.p, cbufs, s);
  } else {
    launch_cholesky_tc(c->blk.p, blist.p, nblk, nblk, ntrow, c->trow.p, c->fac32.p, c->dinv32.p,
                       tc_scratch.p, off, tc_rowblk.p, pmin.p, pfail.p, c->err_flag.p, s);
  }
  c->t_chol_ms = tchol.stop_ms(s);
  // N_KJ = inv(L_KK) L_KJ: a kernel of its own, outside the Cholesky's time
  if (fp64)
    launch_ntransform64(c->blk.p, blist.p, nblk, c->trow.p, c->fac64.p, c->dinv64.p, s);
  else
    launch_ntransform_tc(c->blk.p, nblk, ntrow, c->trow.p, c->fac32.p, c->dinv32.p, tc_rowblk.p,
                         s);
  c->setup_launches += fp64 ? 3 : 4;  // scatter, Cholesky, (block ids,) N transform
  CUDA_TRY(cudaGetLastError());
  std::vector<int32_t> hfail(nblk);
  std::vector<double> hpmin(nblk);
  d2h(hfail.data(), pfail.p, nblk, s);
  d2h(hpmin.data(), pmin.p, nblk, s);
  int32_t hcerr = 0;
  if (cbufs.err.p) d2h(&hcerr, cbufs.err.p, 1, s);
  CUDA_TRY(cudaStreamSynchronize(s));
  if (hcerr) fail(CIMMINO_ETIMEOUT, "a pair wait of the FP64 Cholesky ran out (split block)");
  if (fp64) {
    for (int32_t b = 0; b < nblk; ++b)
      if (hfail[b])
        fail(CIMMINO_ESINGULAR, "Gram block " + std::to_string(b) +
                                    " is not positive definite (A_i is rank deficient)");
  } else {
    // FP64 refactorisation of blocks whose FP32 pivots failed or fell below the ratio
    std::vector<int32_t> fb;
    for (int32_t b = 0; b < nblk; ++b)
      if (hfail[b] || !(hpmin[b] >= c->opts.pivot_ratio_min)) fb.push_back(b);
    c->fallbacks = (int32_t)fb.size();
    if (!fb.empty()) {
      int64_t off64 = 0, doff64 = 0;
      for (int32_t b : fb) {
        BlockDesc &B = c->hblk[b];
        B.prec64 = 1;
        B.dinv_off = doff64;
        doff64 += (int64_t)B.nt * TT;
        for (int32_t I = 0; I < B.nt; ++I) {
          TileRow &R = c->htrow[B.trow0 + I];
          R.off = off64;
          off64 += (int64_t)(I - R.j0 + 1) * TT;
        }
      }
      c->fac64.alloc(off64);
      c->dinv64.alloc(doff64);
      c->factor_bytes += off64 * 8;
      h2d(c->trow.p, c->htrow.data(), ntrow, s);
      h2d(c->blk.p, c->hblk.data(), nblk, s);
      h2d(blist.p, fb.data(), fb.size(), s);
      launch_gram_scatter(c->blk.p, blist.p, (int32_t)fb.size(), c->trow.p, c->brp.p, c->bci.p,
                          c->bcv.p, c->fac64.p, (int64_t)c->fac64.n, 1, s);
      if (maxcta == 0) cholesky_capacity(maxcta, allow_split);
      CholLaunchBufs fbufs;
      run_cholesky64(
          c, plan_cholesky(fb, chol_cost, chol_diag, chol_sync, maxcta, allow_split),
          [&] { return plan_cholesky(fb, chol_cost, chol_diag, chol_sync, maxcta, false); },
          pmin.p, pfail.p, fbufs, s);
      launch_ntransform64(c->blk.p, blist.p, (int32_t)fb.size(), c->trow.p, c->fac64.p,
                          c->dinv64.p, s);
      c->setup_launches += 3;
      d2h(hfail.data(), pfail.p, nblk, s);
      if (fbufs.err.p) d2h(&hcerr, fbufs.err.p, 1, s);
      CUDA_TRY(cudaStreamSynchronize(s));
      if (hcerr) fail(CIMMINO_ETIMEOUT, "a pair wait of the FP64 Cholesky ran out (split block)");
      for (int32_t b : fb)
        if (hfail[b])
          fail(CIMMINO_ESINGULAR, "Gram block " + std::to_string(b) +
                                      " is not positive definite in FP64 (A_i is rank deficient)");
    }
  }
  // ---- transposed copy of every factor, read row-wise by the backward solves
  {
    c->htrowT.resize(ntrow);
    int64_t oT32 = 0, oT64 = 0, ntiles = 0;
    for (const auto &B : c->hblk) {
      for (int32_t I = 0; I < B.nt; ++I) {
        int32_t j1 = I;
        for (int32_t J = I + 1; J < B.nt; ++J)
          if (c->htrow[B.trow0 + J].j0 <= I) j1 = J;
        TileRow &U = c->htrowT[B.trow0 + I];
        U.j0 = j1;
        int64_t &o = B.prec64 ? oT64 : oT32;
        U.off = o;
        o += (int64_t)(j1 - I) * TT;
        // streamed per solve pass: N row, NT row, inv(L_II), inv(L_II)^T
        ntiles += (I - c->htrow[B.trow0 + I].j0) + (j1 - I) + 2;
      }
    }
    // bytes one single-vector solve pass streams: the N and NT rows and the two packed
    // diagonal tiles inv(L_II), inv(L_II)^T of every tile row
    c->pass_bytes = 0;
    for (const auto &B : c->hblk) {
      int64_t t = 0;
      for (int32_t I = 0; I < B.nt; ++I)
        t += (I - c->htrow[B.trow0 + I].j0) + (c->htrowT[B.trow0 + I].j0 - I);
      c->pass_bytes +=
          (t * TT + 2 * (int64_t)B.nt * (B.prec64 ? kPackTile : kBPackTile)) * (B.prec64 ? 8 : 4);
    }
    (void)ntiles;
    // projection launch order: blocks with the most streamed tiles first
    {
      std::vector<int64_t> work(nblk, 0);
      for (int32_t b = 0; b < nblk; ++b) {
        const BlockDesc &B = c->hblk[b];
        for (int32_t I = 0; I < B.nt; ++I)
          work[b] += (I - c->htrow[B.trow0 + I].j0) + (c->htrowT[B.trow0 + I].j0 - I) + 2;
      }
      std::vector<int32_t> order(nblk);
      for (int32_t b = 0; b < nblk; ++b) order[b] = b;
      std::stable_sort(order.begin(), order.end(),
                       [&](int32_t x, int32_t y) { return work[x] > work[y]; });
      c->border.alloc(nblk);
      h2d(c->border.p, order.data(), nblk, s);
      c->hborder = order;
    }
    c->trowT.alloc(ntrow);
    h2d(c->trowT.p, c->htrowT.data(), ntrow, s);
    if (oT32) c->facT32.alloc(oT32);
    if (oT64) c->facT64.alloc(oT64);
    if (c->dinv32.p) {
      c->dinvT32.alloc(c->dinv32.n);
      c->dinvP32.alloc(c->dinv32.n / TT * kBPackTile);
      c->dinvTP32.alloc(c->dinv32.n / TT * kBPackTile);
    }
    if (c->dinv64.p) {
      c->dinvT64.alloc(c->dinv64.n);
      c->dinvP64.alloc(c->dinv64.n / TT * kPackTile);
      c->dinvTP64.alloc(c->dinv64.n / TT * kPackTile);
    }
    FactorPtrs f{c->fac32.p,   c->dinv32.p,   c->facT32.p, c->dinvT32.p,
                 c->fac64.p,   c->dinv64.p,   c->facT64.p, c->dinvT64.p,
                 c->dinvP64.p, c->dinvTP64.p, c->dinvP32.p, c->dinvTP32.p};
    launch_transpose_factor(c->blk.p, nblk, c->trow.p, c->trowT.p, f, s);
    c->setup_launches += 2;  // transposed copies, packed diagonal tiles
  }
  c->t_factor_ms = tfac.stop_ms(s);
  if (!c->opts.keep_aat) {
    c->crp.release();
    c->cci.release();
    c->ccv.release();
    c->have_aat = false;
  }
  stage.next("cimmino.setup.tables");
  // ---- vector-kernel CTA table (kVecRows rows per CTA, never straddling systems) and
  // the 32-row slices of the sliced-ELL copies of A and A^T
  std::vector<int64_t> hsrow0;
  std::vector<int32_t> hsrows;
  for (int32_t q = 0; q < nsys; ++q) {
    SysDesc &S = c->hsys[q];
    S.cta0 = (int32_t)c->hcta.size();
    for (int64_t r = 0; r < S.n; r += kVecRows) {
      CtaDesc C{};
      C.row0 = S.row0 + r;
      C.rows = (int32_t)std::min<int64_t>(kVecRows, S.n - r);
      C.sys = q;
      C.slice0 = (int32_t)hsrow0.size();
      for (int64_t r2 = r; r2 < r + C.rows; r2 += 32) {
        hsrow0.push_back(S.row0 + r2);
        hsrows.push_back((int32_t)std::min<int64_t>(32, S.n - r2));
      }
      c->hcta.push_back(C);
    }
    S.ncta = (int32_t)c->hcta.size() - S.cta0;
  }
  {
    const int32_t ns = (int32_t)hsrow0.size();
    DBuf<int64_t> srow0, scnt;
    DBuf<int32_t> srows;
    srow0.alloc(ns);
    srows.alloc(ns);
    scnt.alloc(ns);
    h2d(srow0.p, hsrow0.data(), ns, s);
    h2d(srows.p, hsrows.data(), ns, s);
    auto build = [&](const int64_t *ptr, const int32_t *idx, const double *val,
                     const int32_t *rmap, DBuf<int64_t> &off, DBuf<int32_t> &col,
                     DBuf<double> &vv) {
      off.alloc(ns + 1);
      sell_rows_width(ptr, srow0.p, srows.p, ns, rmap, scnt.p, s);
      launch_scan_counts(scnt.p, off.p, ns, tmp.p, tl, s);
      int64_t tot = 0;
      d2h(&tot, off.p + ns, 1, s);
      CUDA_TRY(cudaStreamSynchronize(s));
      col.alloc(tot);
      vv.alloc(tot);
      sell_rows_fill(ptr, idx, val, srow0.p, srows.p, ns, rmap, off.p, col.p, vv.p, s);
      c->setup_launches += 5;  // widths, 3-pass scan, fill
    };
    c->cta.alloc(c->hcta.size());
    h2d(c->cta.p, c->hcta.data(), c->hcta.size(), s);
    build(c->rp.p, c->ci.p, c->va.p, nullptr, c->aoff, c->acol, c->aval);
    // A^T's rows (the columns of A) vary in length: inside every CTA's chunk they are
    // ordered by decreasing length, so its 32-row slices pad little
    c->tord.alloc(N);
    chunk_order(c->cp.p, c->cta.p, (int32_t)c->hcta.size(), c->tord.p, s);
    c->setup_launches += 1;
    build(c->cp.p, c->ri.p, c->cv.p, c->tord.p, c->toff, c->tcol, c->tval);
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  c->sys.alloc(nsys);
  h2d(c->sys.p, c->hsys.data(), nsys, s);
  c->rowabs.alloc(N);
  launch_row_abs(c->rp.p, c->ci.p, c->va.p, c->d.p, c->cs.p, N, c->rowabs.p, s);
  c->setup_launches += 1;
  // projection ring: as many factor-tile slots as fit beside the block vectors
  bool any64 = false;
  for (const auto &B : c->hblk) any64 |= B.prec64 != 0;
  c->proj_slot_bytes = kTile * kTile * (any64 ? 8 : 4);
  c->proj_wbytes = any64 ? 8 : 4;
  c->proj_slots =
      std::min(kMaxProjSlots, (kProjSmemMax - proj_smem_bytes(c->max_mp, 0, 0, c->proj_wbytes)) /
                                  c->proj_slot_bytes);
  if (c->proj_slots < 2) fail(CIMMINO_EUNSUPPORTED, "block too large for the projection kernel");
  c->proj_smem = proj_smem_bytes(c->max_mp, c->proj_slots, c->proj_slot_bytes, c->proj_wbytes);
  c->proj_minb = 1;
  CUDA_TRY(set_proj_smem_attr(c->proj_smem));
  if (!c->err_flag.p) c->err_flag.alloc(1);
  CUDA_TRY(cudaMemsetAsync(c->err_flag.p, 0, sizeof(int32_t), s));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ projection autotuner
// The projection kernel's free parameters: the depth of its factor-tile ring and whether
// its registers are budgeted for one or two CTAs per SM (a second block then fills the
// first one's chain barriers, at the price of a shallower ring).  Candidates are timed on
// the context's own blocks (a few launches on a fixed vector) and the fastest is kept; with
// opts.tune_cache the choice is stored per (GPU, precision, block shape) and reused.
struct ProjConfig {
  int32_t minb, slots;
};

std::string tune_key(const cimmino_ctx *c) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, c->device);
  int64_t tiles = 0;
  for (const auto &B : c->hblk)
    for (int32_t I = 0; I < B.nt; ++I)
      tiles += (I - c->htrow[B.trow0 + I].j0) + (c->htrowT[B.trow0 + I].j0 - I) + 2;
  std::string name(prop.name);
  for (char &ch : name)
    if (ch == ' ' || ch == '|') ch = '_';
  return name + "|" + (c->proj_wbytes == 8 ? "fp64" : "fp32") + "|mp" +
         std::to_string(c->max_mp) + "|blocks" + std::to_string(c->hblk.size()) + "|tiles" +
         std::to_string(tiles);
}

bool tune_cache_read(const char *path, const std::string &key, ProjConfig &cfg) {
  if (!path) return false;
  FILE *f = std::fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    char k[400];
    int minb = 0, slots = 0;
    if (std::sscanf(line, "%399s %d %d", k, &minb, &slots) == 3 && key == k &&
        (minb == 1 || minb == 2) && slots >= 2 && slots <= kMaxProjSlots) {
      cfg = {minb, slots};
      found = true;  // the last entry for a key wins
    }
  }
  std::fclose(f);
  return found;
}

void tune_cache_write(const char *path, const std::string &key, const ProjConfig &cfg) {
  if (!path) return;
  FILE *f = std::fopen(path, "a");
  if (!f) return;  // an unwritable cache only costs a re-tune next time
  std::fprintf(f, "%s %d %d\n", key.c_str(), cfg.minb, cfg.slots);
  std::fclose(f);
}

__global__ void k_fill(double *v, int64_t n, double x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = x;
}

void apply_proj_config(cimmino_ctx *c, const ProjConfig &cfg) {
  c->proj_minb = cfg.minb;
  c->proj_slots = cfg.slots;
  c->proj_smem = proj_smem_bytes(c->max_mp, c->proj_slots, c->proj_slot_bytes, c->proj_wbytes);
  CUDA_TRY(set_proj_smem_attr(c->proj_smem));
  c->args.proj_minb = c->proj_minb;
  c->args.proj_slots = c->proj_slots;
  c->args.proj_smem = c->proj_smem;
}

void ensure_solve_buffers(cimmino_ctx *c, int32_t nrhs);

void tune_projection(cimmino_ctx *c) {
  const std::string key = tune_key(c);
  ProjConfig best{c->proj_minb, c->proj_slots};
  if (tune_cache_read(c->opts.tune_cache, key, best)) {
    ensure_solve_buffers(c, 1);
    apply_proj_config(c, best);
    c->tuned = 2;
    return;
  }
  ensure_solve_buffers(c, 1);
  cudaStream_t s = c->stream;
  const int64_t N = c->N;
  k_fill<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(c->u.p, N, 1.0);
  std::vector<ProjConfig> cand;
  const int base = proj_smem_bytes(c->max_mp, 0, 0, c->proj_wbytes);
  const int max1 = std::min(kMaxProjSlots, (kProjSmemMax - base) / c->proj_slot_bytes);
  cand.push_back({1, max1});
  if (max1 > 8) cand.push_back({1, 8});
  // two CTAs per SM: half of the SM's shared memory each (less the static part)
  const int max2 = std::min(kMaxProjSlots, (kProjSmemMax / 2 - 2048 - base) / c->proj_slot_bytes);
  if (max2 >= 2) cand.push_back({2, max2});
  Timer tm;
  double best_ms = 1e300;
  for (const ProjConfig &cfg : cand) {
    apply_proj_config(c, cfg);
    launch_proj(c->args, c->u.p, c->y.p, 0, s);  // warm-up
    tm.start(s);
    constexpr int kReps = 3;
    for (int r = 0; r < kReps; ++r) launch_proj(c->args, c->u.p, c->y.p, 0, s);
    CUDA_TRY(cudaGetLastError());
    const double ms = tm.stop_ms(s) / kReps;
    if (ms < best_ms) {
      best_ms = ms;
      best = cfg;
    }
  }
  apply_proj_config(c, best);
  c->tuned = 1;
  tune_cache_write(c->opts.tune_cache, key, best);
}

// ------------------------------------------------------------------ solve
void ensure_solve_buffers(cimmino_ctx *c, int32_t nrhs) {
  if (c->nrhs == nrhs) return;
  AllocScope scope(&c->mem);
  const int64_t N = c->N;
  const int64_t V = N * nrhs;
  c->lane.alloc((size_t)c->nsys * nrhs);
  c->fs.alloc(V);
  c->x.alloc(V);
  c->p.alloc(V);
  c->r.alloc(V);
  c->psi.alloc(V);
  c->u.alloc(V);
  c->y.alloc(V);
  c->Fin.alloc(V);
  c->part.alloc((size_t)4 * c->hcta.size() * nrhs);
  c->stats4.alloc((size_t)4 * c->hcta.size() * nrhs);
  c->cnt.alloc((size_t)4 * c->nsys);
  c->refine_total.alloc(1);
  c->refine_max.alloc(1);
  c->nrhs = nrhs;
  IterArgs &a = c->args;
  a.rp = c->rp.p;
  a.ci = c->ci.p;
  a.va = c->va.p;
  a.cp = c->cp.p;
  a.ri = c->ri.p;
  a.cv = c->cv.p;
  a.d = c->d.p;
  a.cs = c->cs.p;
  a.brp = c->brp.p;
  a.bci = c->bci.p;
  a.bcv = c->bcv.p;
  a.aoff = c->aoff.p;
  a.acol = c->acol.p;
  a.aval = c->aval.p;
  a.toff = c->toff.p;
  a.tord = c->tord.p;
  a.tcol = c->tcol.p;
  a.tval = c->tval.p;
  a.soff = c->soff.p;
  a.scol = c->scol.p;
  a.sval = c->sval.p;
  a.blk = c->blk.p;
  a.border = c->border.p;
  a.trow = c->trow.p;
  a.trowT = c->trowT.p;
  a.fac32 = c->fac32.p;
  a.dinv32 = c->dinv32.p;
  a.facT32 = c->facT32.p;
  a.dinvT32 = c->dinvT32.p;
  a.fac64 = c->fac64.p;
  a.dinv64 = c->dinv64.p;
  a.facT64 = c->facT64.p;
  a.dinvT64 = c->dinvT64.p;
  a.dinvP32 = c->dinvP32.p;
  a.dinvTP32 = c->dinvTP32.p;
  a.dinvP64 = c->dinvP64.p;
  a.dinvTP64 = c->dinvTP64.p;
  a.sys = c->sys.p;
  a.cta = c->cta.p;
  a.lane = c->lane.p;
  a.fs = c->fs.p;
  a.x = c->x.p;
  a.p = c->p.p;
  a.r = c->r.p;
  a.psi = c->psi.p;
  a.u = c->u.p;
  a.y = c->y.p;
  a.part = c->part.p;
  a.cnt = c->cnt.p;
  a.refine_total = c->refine_total.p;
  a.refine_max = c->refine_max.p;
  a.N = N;
  a.nsys = c->nsys;
  a.ncta = (int32_t)c->hcta.size();
  a.nblk = (int32_t)c->hblk.size();
  a.nrhs = nrhs;
  a.refine_steps = c->opts.precision == CIMMINO_FP32_REFINE ? c->opts.refine_max : 0;
  a.refine_tol = c->opts.refine_tol;
  a.refine_relax = c->opts.refine_relax;
  a.max_iter = c->opts.max_iter;
  a.max_mp = c->max_mp;
  a.proj_smem = c->proj_smem;
  a.proj_slots = c->proj_slots;
  a.proj_minb = c->proj_minb;
  a.proj_slot_bytes = c->proj_slot_bytes;
  a.proj_wbytes = c->proj_wbytes;
  // several right-hand sides: groups of 16 (FP32 factors) or 8 share each factor tile,
  // as long as the group's vectors and a ring of at least 2 slots fit in shared memory
  a.proj_rg = 0;
  a.proj_mr_slots = 0;
  a.proj_mr_smem = 0;
  if (nrhs > 1 && c->opts.multi_rhs) {
    for (int rg = (c->proj_wbytes == 4 && nrhs > 8) ? 16 : 8; rg >= 8; rg /= 2) {
      // the multi-RHS kernel has up to 2 KB of static shared memory besides this
      const int budget = kProjSmemMax - 2048;
      const int base = proj_mr_smem_bytes(c->max_mp, rg, 0, c->proj_slot_bytes, c->proj_wbytes);
      const int slots = std::min(kMaxProjSlots, (budget - base) / c->proj_slot_bytes);
      if (base < budget && slots >= 2) {
        a.proj_rg = rg;
        a.proj_mr_slots = slots;
        a.proj_mr_smem = base + slots * c->proj_slot_bytes;
        CUDA_TRY(set_proj_mr_smem_attr(rg, a.proj_mr_smem));
        break;
      }
    }
  }
  // with opts.multi_rhs == 2, FP32 blocks of up to 32 tile rows take the tensor-core kernel
  // and the others (FP64 fallbacks, larger blocks) the CUDA-core one, in one launch each
  const int32_t nblk = (int32_t)c->hblk.size();
  std::vector<int32_t> ml = c->hborder;
  c->mr_ntc = 0;
  if (a.proj_rg > 0 && c->opts.multi_rhs == 2 && c->fac32.p && c->dinv32.p) {
    std::vector<int32_t> tc, rest;
    for (int32_t b : c->hborder) {
      const BlockDesc &B = c->hblk[b];
      (B.prec64 == 0 && B.nt <= proj_mr_tc_max_tiles() ? tc : rest).push_back(b);
    }
    const size_t mb = tile_map_bytes();
    c->tmaps.assign(4 * mb, 0);
    // the transposed factor is empty when no block has an off-diagonal tile: its map is
    // then never read, and any valid array stands in
    const float *ft = c->facT32.p ? c->facT32.p : c->dinv32.p;
    const int64_t nft = c->facT32.p ? (int64_t)c->facT32.n : (int64_t)c->dinv32.n;
    if (!tc.empty() && make_tile_map(&c->tmaps[0], c->fac32.p, (int64_t)c->fac32.n) &&
        make_tile_map(&c->tmaps[mb], ft, nft) &&
        make_tile_map(&c->tmaps[2 * mb], c->dinv32.p, (int64_t)c->dinv32.n) &&
        make_tile_map(&c->tmaps[3 * mb], c->dinvT32.p, (int64_t)c->dinvT32.n)) {
      CUDA_TRY(set_proj_mr_tc_smem_attr());
      ml = tc;
      ml.insert(ml.end(), rest.begin(), rest.end());
      c->mr_ntc = (int32_t)tc.size();
    }
  }
  c->mr_list.alloc(nblk);
  h2d(c->mr_list.p, ml.data(), nblk, c->stream);
  a.mr_list = c->mr_list.p;
  a.mr_ntc = c->mr_ntc;
  a.mr_tmaps = c->tmaps.empty() ? nullptr : c->tmaps.data();
  a.err = c->err_flag.p;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
}

// Fin ([nrhs][N], original row order) must be filled by the caller.
int solve_impl(cimmino_ctx *c, int32_t nrhs, double tol, cimmino_stats *stats) {
  cudaStream_t s = c->stream;
  IterArgs &a = c->args;
  a.tol = tol;
  Stages stage("cimmino.solve.xi");
  Timer tsolve;
  tsolve.start(s);
  CUDA_TRY(cudaMemsetAsync(c->cnt.p, 0, sizeof(int32_t) * 4 * c->nsys, s));
  CUDA_TRY(cudaMemsetAsync(c->refine_total.p, 0, sizeof(int64_t), s));
  CUDA_TRY(cudaMemsetAsync(c->refine_max.p, 0, sizeof(int32_t), s));
  CUDA_TRY(cudaMemsetAsync(c->lane.p, 0, sizeof(LaneState) * c->nsys * nrhs, s));
  launch_rhs_scale(a, c->Fin.p, c->perm.p, s);
  // xi = sum_i A_i^+ f_i, then r = p = xi, x = 0
  launch_proj(a, c->fs.p, c->y.p, 0, s);
  launch_spmv_t(a, c->y.p, c->psi.p, s);
  launch_cg_init(a, s);
  CUDA_TRY(cudaGetLastError());
  stage.next("cimmino.solve.cg");
  const int32_t G = c->opts.check_every;
  const int32_t nl = c->nsys * nrhs;
  std::vector<LaneState> hl(nl);
  int64_t launched = 0;
  const bool timing = c->opts.time_proj != 0;
  std::vector<double> iter_ms;  // live projection time per iteration (timing only)
  bool timing_ok = timing;
  if (timing && c->pev.size() != (size_t)2 * G) {
    for (cudaEvent_t e : c->pev) cudaEventDestroy(e);
    c->pev.assign((size_t)2 * G, nullptr);
    for (auto &e : c->pev) CUDA_TRY(cudaEventCreate(&e));
  }
  auto ev = [&](int32_t i, int which) -> cudaEvent_t {
    return timing ? c->pev[(size_t)2 * i + which] : nullptr;
  };
  const int64_t limit = (int64_t)c->opts.max_iter + 2 * G + 2;
  for (;;) {
    // timed solves launch eagerly: events recorded inside a captured graph are internal
    // to it and cannot be timed
    if (c->opts.use_graph && !timing) {
      if (!c->graph || c->graph_nrhs != nrhs || c->graph_iters != G) {
        if (c->graph) cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
        cudaGraph_t g;
        CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int32_t i = 0; i < G; ++i) launch_iteration(a, s);
        CUDA_TRY(cudaStreamEndCapture(s, &g));
        cudaError_t e = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        CUDA_TRY(e);
        c->graph_nrhs = nrhs;
        c->graph_iters = G;
      }
      CUDA_TRY(cudaGraphLaunch(c->graph, s));
    } else {
      for (int32_t i = 0; i < G; ++i) launch_iteration(a, s, ev(i, 0), ev(i, 1));
      CUDA_TRY(cudaGetLastError());
    }
    launched += G;
    d2h(hl.data(), c->lane.p, nl, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int32_t i = 0; timing_ok && i < G; ++i) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, c->pev[(size_t)2 * i], c->pev[(size_t)2 * i + 1]) !=
          cudaSuccess) {
        cudaGetLastError();  // timing unavailable: report none, the solve goes on
        timing_ok = false;
      }
      iter_ms.push_back(ms);
    }
    bool running = false;
    for (const auto &L : hl) running |= (L.status == CIMMINO_RUNNING);
    if (!running) break;
    if (launched > limit) fail(CIMMINO_ETIMEOUT, "CG lanes still running past max_iter");
  }
  stage.next("cimmino.solve.stats");
  // backward error gamma (Eq. 3.1) per lane
  launch_final_stats(a, c->Fin.p, c->rowabs.p, c->stats4.p, s);
  // the CG iterate lives in the column-scaled space y = diag(cs) x
  if (a.cs) launch_unscale_cols(c->x.p, a.cs, c->N, nrhs, s);
  // live projection time: the iterations in which some lane still ran its projection
  c->proj_ms_total = 0.0;
  c->proj_launches = -1;
  if (timing_ok) {
    int64_t nrun = 0;
    for (const auto &L : hl) nrun = std::max<int64_t>(nrun, L.iters);
    nrun = std::min<int64_t>(nrun, (int64_t)iter_ms.size());
    for (int64_t t = 0; t < nrun; ++t) c->proj_ms_total += iter_ms[(size_t)t];
    c->proj_launches = nrun;
  }
  std::vector<double> h4((size_t)4 * c->hcta.size() * nrhs);
  d2h(h4.data(), c->stats4.p, h4.size(), s);
  int64_t rtot = 0;
  int32_t rmax = 0;
  d2h(&rtot, c->refine_total.p, 1, s);
  d2h(&rmax, c->refine_max.p, 1, s);
  int32_t herr = 0;
  d2h(&herr, c->err_flag.p, 1, s);
  const double tms = tsolve.stop_ms(s);
  CUDA_TRY(cudaGetLastError());
  if (herr)
    fail(CIMMINO_ETIMEOUT, "a bounded wait ran out (error word " + std::to_string(herr) +
                               ": 1/2 projection ring, 4 Cholesky MMA)");
  int ret = CIMMINO_OK;
  for (int32_t q = 0; q < c->nsys; ++q) {
    const SysDesc &S = c->hsys[q];
    for (int32_t k = 0; k < nrhs; ++k) {
      const LaneState &L = hl[q * nrhs + k];
      double rinf = 0, x1 = 0, finf = 0, ainf = 0;
      for (int32_t cc = S.cta0; cc < S.cta0 + S.ncta; ++cc) {
        const double *o = &h4[((size_t)cc * nrhs + k) * 4];
        rinf = std::max(rinf, o[0]);
        x1 += o[1];
        finf = std::max(finf, o[2]);
        ainf = std::max(ainf, o[3]);
      }
      int st = L.status == CIMMINO_CONVERGED ? CIMMINO_OK : L.status;
      if (st != CIMMINO_OK && ret == CIMMINO_OK) ret = st;
      if (stats) {
        cimmino_stats &o = stats[q * nrhs + k];
        o.status = st;
        o.iters = L.iters;
        o.rel_res = L.relres;
        double den = ainf * x1 + finf;
        o.backward_err = den > 0 ? rinf / den : 0.0;
        o.refine_steps_total = rtot;
        o.refine_steps_max = rmax;
        o.fallbacks = c->fallbacks;
        o.t_setup_ms = c->t_setup_ms;
        o.t_factor_ms = c->t_factor_ms;
        o.t_solve_ms = tms;
        o.nnz_aat = c->nnzc;
        o.factor_bytes = c->factor_bytes;
        o.factor_flops = c->factor_flops;
        o.t_chol_ms = c->t_chol_ms;
        o.nnz_gram = c->nnz_bd;
        o.proj_slots = c->proj_slots;
        o.proj_ctas_per_sm = c->proj_minb;
        o.proj_tuned = c->tuned;
        o.mr_tc_blocks = nrhs > 1 ? c->mr_ntc : 0;
        o.chol_split_blocks = c->chol_split;
        o.pass_bytes = c->pass_bytes;
        // rhs scale, xi projection, A^T y, CG init, 4 kernels plus the projection per
        // iteration, final stats; several right-hand sides may take two projection kernels
        const int pk = (nrhs > 1 && c->mr_ntc > 0 && c->mr_ntc < (int32_t)c->hblk.size()) ? 2 : 1;
        o.kernel_launches = c->setup_launches + 4 + pk + (4 + pk) * launched +
                            (nrhs > 1 ? 1 : 0) + (a.cs ? 1 : 0);
      }
    }
  }
  return ret;
}

// Message of the first failing right-hand side (its status code) of a solve.
const char *lane_failure_message(int code) {
  switch (code) {
    case CIMMINO_ENOCONV:
      return "max_iter reached before convergence";
    case CIMMINO_EINVAL:
      return "a right-hand side holds NaN or Inf";
    case CIMMINO_EUNSUPPORTED:
      return "the squared 2-norm of a right-hand side overflows FP64 (entries above about "
             "1e154)";
    default:
      return "CG breakdown (p^T H p <= 0 or not finite)";
  }
}

int set_error(cimmino_ctx *c, const Error &e) {
  if (c)
    c->err = e.msg;
  else
    g_last_error = e.msg;
  g_last_error = e.msg;
  return e.code;
}

}  // namespace

void cimmino::record_last_error(const std::string &msg) { g_last_error = msg; }

// ====================================================================== C ABI
extern "C" {

void cimmino_opts_default(cimmino_opts *opts) {
  if (opts) opts_default(opts);
}

const char *cimmino_version(void) { return "cimmino-gb300 1.0 (sm_103a)"; }

int cimmino_setup_batch(int32_t nsys, const cimmino_csr *A, const int32_t *K,
                        const int32_t *const *perm, const int64_t *const *block_ptr,
                        const cimmino_opts *opts, cimmino_ctx **out) {
  if (out) *out = nullptr;
  if (!out || !A || !K || !block_ptr || nsys < 1) {
    g_last_error = "invalid argument (NULL pointer or nsys < 1)";
    return CIMMINO_EINVAL;
  }
  cimmino_ctx *c = new (std::nothrow) cimmino_ctx();
  if (!c) return CIMMINO_ENOMEM;
  try {
    if (opts)
      c->opts = *opts;
    else
      opts_default(&c->opts);
    check_opts(c->opts);
    CUDA_TRY(cudaGetDevice(&c->device));
    if (c->opts.stream) {
      c->stream = static_cast<cudaStream_t>(c->opts.stream);
    } else {
      CUDA_TRY(cudaStreamCreateWithFlags(&c->owned.s, cudaStreamNonBlocking));
      c->stream = c->owned.s;
      c->own_stream = true;
    }
    c->mem.fa = c->opts.alloc;
    c->mem.ff = c->opts.free;
    c->mem.user = c->opts.alloc_user;
    c->mem.stream = c->stream;
    AllocScope scope(&c->mem);
    setup_impl(c, nsys, A, K, perm, block_ptr);
    if (c->opts.tune) tune_projection(c);
  } catch (const Error &e) {
    int code = set_error(nullptr, e);
    if (c->stream) cudaStreamSynchronize(c->stream);
    delete c;
    return code;
  }
  *out = c;
  return CIMMINO_OK;
}

int cimmino_setup(const cimmino_csr *A, int32_t K, const int32_t *perm, const int64_t *block_ptr,
                  const cimmino_opts *opts, cimmino_ctx **out) {
  const int32_t *pa[1] = {perm};
  const int64_t *ba[1] = {block_ptr};
  if (!block_ptr) {
    if (out) *out = nullptr;
    g_last_error = "block_ptr is NULL";
    return CIMMINO_EINVAL;
  }
  return cimmino_setup_batch(1, A, &K, pa, ba, opts, out);
}

void cimmino_free(cimmino_ctx *ctx) {
  if (!ctx) return;
  int cur = 0;
  const int dev = ctx->device;
  cudaGetDevice(&cur);
  if (cur != dev) cudaSetDevice(dev);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  delete ctx;
  if (cur != dev) cudaSetDevice(cur);
}

const char *cimmino_last_error(const cimmino_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_last_error.c_str();
}

int cimmino_solve(cimmino_ctx *ctx, const double *F, int32_t nrhs, int64_t ld, double tol,
                  double *X, int32_t on_device, cimmino_stats *stats) {
  if (!ctx) return CIMMINO_EINVAL;
  try {
    if (ctx->nsys != 1) fail(CIMMINO_EINVAL, "cimmino_solve needs a single-system context");
    if (!F || !X || nrhs < 1 || ld < ctx->N) fail(CIMMINO_EINVAL, "bad F / X / nrhs / ld");
    if (!(tol > 0.0)) fail(CIMMINO_EINVAL, "tol must be > 0");
    (void)on_device;  // copies use unified addressing, host or device alike
    ensure_solve_buffers(ctx, nrhs);
    cudaStream_t s = ctx->stream;
    const int64_t N = ctx->N;
    CUDA_TRY(cudaMemcpy2DAsync(ctx->Fin.p, N * sizeof(double), F, ld * sizeof(double),
                               N * sizeof(double), nrhs, cudaMemcpyDefault, s));
    int ret = solve_impl(ctx, nrhs, tol, stats);
    if (nrhs == 1) {
      CUDA_TRY(cudaMemcpyAsync(X, ctx->x.p, N * sizeof(double), cudaMemcpyDefault, s));
    } else {
      int64_t tot = N * nrhs;
      k_interleave_to_cols<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ctx->x.p, N, nrhs,
                                                                         ctx->Fin.p);
      CUDA_TRY(cudaMemcpy2DAsync(X, ld * sizeof(double), ctx->Fin.p, N * sizeof(double),
                                 N * sizeof(double), nrhs, cudaMemcpyDefault, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    if (ret != CIMMINO_OK) ctx->err = lane_failure_message(ret);
    return ret;
  } catch (const Error &e) {
    return set_error(ctx, e);
  }
}

int cimmino_solve_batch(cimmino_ctx *ctx, const double *const *F, double tol, double *const *X,
                        int32_t on_device, cimmino_stats *stats) {
  if (!ctx) return CIMMINO_EINVAL;
  try {
    if (!F || !X) fail(CIMMINO_EINVAL, "F / X is NULL");
    if (!(tol > 0.0)) fail(CIMMINO_EINVAL, "tol must be > 0");
    (void)on_device;
    ensure_solve_buffers(ctx, 1);
    cudaStream_t s = ctx->stream;
    for (int32_t q = 0; q < ctx->nsys; ++q) {
      if (!F[q] || !X[q]) fail(CIMMINO_EINVAL, "F[s] / X[s] is NULL");
      h2d(ctx->Fin.p + ctx->hsys[q].row0, F[q], ctx->hsys[q].n, s);
    }
    int ret = solve_impl(ctx, 1, tol, stats);
    for (int32_t q = 0; q < ctx->nsys; ++q)
      d2h(X[q], ctx->x.p + ctx->hsys[q].row0, ctx->hsys[q].n, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    if (ret != CIMMINO_OK) ctx->err = lane_failure_message(ret);
    return ret;
  } catch (const Error &e) {
    return set_error(ctx, e);
  }
}

int cimmino_get_aat_nnz(cimmino_ctx *ctx, int64_t *nnz) {
  if (!ctx || !nnz) return CIMMINO_EINVAL;
  if (!ctx->have_aat) {
    ctx->err = "C = A A^T was not kept (set opts.keep_aat = 1)";
    return CIMMINO_EINVAL;
  }
  *nnz = ctx->nnzc;
  return CIMMINO_OK;
}

int cimmino_get_aat(cimmino_ctx *ctx, int64_t *row_ptr, int32_t *col_idx, double *val) {
  if (!ctx || !row_ptr || !col_idx || !val) return CIMMINO_EINVAL;
  if (!ctx->have_aat) {
    ctx->err = "C = A A^T was not kept (set opts.keep_aat = 1)";
    return CIMMINO_EINVAL;
  }
  try {
    cudaStream_t s = ctx->stream;
    d2h(row_ptr, ctx->crp.p, ctx->N + 1, s);
    d2h(col_idx, ctx->cci.p, ctx->nnzc, s);
    d2h(val, ctx->ccv.p, ctx->nnzc, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    return CIMMINO_OK;
  } catch (const Error &e) {
    return set_error(ctx, e);
  }
}

int cimmino_fp64_peak(double *tflops) {
  if (!tflops) {
    g_last_error = "invalid argument (NULL tflops)";
    return CIMMINO_EINVAL;
  }
  try {
    OwnedStream os;
    CUDA_TRY(cudaStreamCreateWithFlags(&os.s, cudaStreamNonBlocking));
    Allocator mem;
    mem.stream = os.s;
    AllocScope scope(&mem);
    DBuf<double> sink;
    sink.alloc(1);
    Timer tm;
    int64_t fmas = 0;
    const double ms = launch_dfma_probe(1 << 14, sink.p, os.s, tm.a, tm.b, &fmas);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(os.s));
    if (!(ms > 0.0)) fail(CIMMINO_ECUDA, "the probe's timing failed");
    *tflops = 2.0 * (double)fmas / (ms * 1e-3) / 1e12;
    return CIMMINO_OK;
  } catch (const Error &e) {
    return set_error(nullptr, e);
  }
}

int cimmino_cholesky_schedule(int32_t nblk, const int32_t *nt, const int64_t *ntrsm,
                              const int64_t *nfull, int32_t maxcta, int32_t allow_split,
                              int32_t *ncta, int32_t *cta_ptr, int32_t *items, int32_t *nsplit,
                              double *makespan) {
  if (nblk < 0 || maxcta < 1 || (nblk > 0 && (!nt || !ntrsm || !nfull || !items)) || !ncta ||
      !cta_ptr || !nsplit || !makespan) {
    g_last_error = "nblk >= 0, maxcta >= 1 and non-NULL arrays required";
    return CIMMINO_EINVAL;
  }
  try {
    std::vector<double> cost(nblk), diag(nblk), sync(nblk);
    std::vector<int32_t> blocks(nblk);
    for (int32_t b = 0; b < nblk; ++b) {
      if (nt[b] < 1 || ntrsm[b] < 0 || nfull[b] < 0) {
        g_last_error = "block " + std::to_string(b) + ": nt >= 1, ntrsm >= 0, nfull >= 0 required";
        return CIMMINO_EINVAL;
      }
      chol_block_cost(nt[b], ntrsm[b], nfull[b], cost[b], diag[b], sync[b]);
      blocks[b] = b;
    }
    const CholPlan P = plan_cholesky(blocks, cost, diag, sync, maxcta, allow_split != 0);
    *ncta = (int32_t)P.ptr.size() - 1;
    for (size_t k = 0; k < P.ptr.size(); ++k) cta_ptr[k] = P.ptr[k];
    for (size_t q = 0; q < P.items.size(); ++q) {
      items[3 * q] = P.items[q].b;
      items[3 * q + 1] = P.items[q].part;
      items[3 * q + 2] = P.items[q].nparts;
    }
    *nsplit = P.nsplit;
    *makespan = P.makespan;
    return CIMMINO_OK;
  } catch (const std::bad_alloc &) {
    g_last_error = "out of host memory";
    return CIMMINO_ENOMEM;
  }
}

int cimmino_selftest_wait(int32_t limit_us, int32_t *err_word) {
  if (limit_us < 1 || limit_us > 1000000 || !err_word) {
    g_last_error = "limit_us must be in [1, 1e6] and err_word non-NULL";
    return CIMMINO_EINVAL;
  }
  try {
    OwnedStream os;  // destroyed after the buffer below has been returned
    CUDA_TRY(cudaStreamCreateWithFlags(&os.s, cudaStreamNonBlocking));
    const cudaStream_t s = os.s;
    Allocator mem;
    mem.stream = s;
    AllocScope scope(&mem);
    DBuf<int32_t> err, flag;
    err.alloc(1);
    flag.alloc(2);
    cudaError_t e = cudaMemsetAsync(err.p, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag.p, 0, 2 * sizeof(int32_t), s);
    if (e == cudaSuccess) {
      launch_wait_selftest((uint64_t)limit_us * 1000ull, err.p, s);
      launch_pair_selftest((uint64_t)limit_us * 1000ull, flag.p, err.p, s);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(err_word, err.p, sizeof(int32_t), cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    CUDA_TRY(e);
    if (*err_word) {
      g_last_error = "the self-test wait ran out of its budget (error word " +
                     std::to_string(*err_word) + ")";
      return CIMMINO_ETIMEOUT;
    }
    return CIMMINO_OK;
  } catch (const Error &e) {
    return set_error(nullptr, e);
  }
}

int cimmino_proj_timing(cimmino_ctx *ctx, double *ms_total, int64_t *launches) {
  if (!ctx || !ms_total || !launches) return CIMMINO_EINVAL;
  if (!ctx->opts.time_proj || ctx->proj_launches < 0) {
    ctx->err = "no projection timing: set opts.time_proj = 1 and solve first";
    return CIMMINO_EINVAL;
  }
  *ms_total = ctx->proj_ms_total;
  *launches = ctx->proj_launches;
  return CIMMINO_OK;
}

int cimmino_get_colscale(cimmino_ctx *ctx, double *cs) {
  if (!ctx || !cs) return CIMMINO_EINVAL;
  try {
    if (!ctx->cs.p) {
      for (int64_t j = 0; j < ctx->N; ++j) cs[j] = 1.0;
      return CIMMINO_OK;
    }
    d2h(cs, ctx->cs.p, ctx->N, ctx->stream);
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return CIMMINO_OK;
  } catch (const Error &e) {
    return set_error(ctx, e);
  }
}

int cimmino_get_scaled(cimmino_ctx *ctx, int64_t *row_ptr, int32_t *col_idx, double *val,
                       double *d) {
  if (!ctx || !row_ptr || !col_idx || !val || !d) return CIMMINO_EINVAL;
  try {
    cudaStream_t s = ctx->stream;
    d2h(row_ptr, ctx->rp.p, ctx->N + 1, s);
    d2h(col_idx, ctx->ci.p, ctx->nnz, s);
    d2h(val, ctx->va.p, ctx->nnz, s);
    d2h(d, ctx->d.p, ctx->N, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    return CIMMINO_OK;
  } catch (const Error &e) {
    return set_error(ctx, e);
  }
}

int cimmino_block_rows(cimmino_ctx *ctx, int32_t b, int32_t *m) {
  if (!ctx || !m || b < 0 || b >= (int32_t)ctx->hblk.size()) return CIMMINO_EINVAL;
  *m = ctx->hblk[b].m;
  return CIMMINO_OK;
}

int cimmino_get_factor(cimmino_ctx *ctx, int32_t b, double *L, int32_t *is_fp64) {
  if (!ctx || !L || b < 0 || b >= (int32_t)ctx->hblk.size()) return CIMMINO_EINVAL;
  try {
    const BlockDesc &B = ctx->hblk[b];
    const int64_t TT = (int64_t)kTile * kTile;
    const TileRow &first = ctx->htrow[B.trow0];
    const TileRow &last = ctx->htrow[B.trow0 + B.nt - 1];
    const int64_t span = last.off + (int64_t)(B.nt - 1 - last.j0 + 1) * TT - first.off;
    std::vector<double> buf(span);
    cudaStream_t s = ctx->stream;
    if (B.prec64) {
      d2h(buf.data(), ctx->fac64.p + first.off, span, s);
    } else {
      std::vector<float> f(span);
      d2h(f.data(), ctx->fac32.p + first.off, span, s);
      CUDA_TRY(cudaStreamSynchronize(s));
      for (int64_t i = 0; i < span; ++i) buf[i] = f[i];
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    const int m = B.m;
    std::memset(L, 0, sizeof(double) * (size_t)m * m);
    // stored: diagonal tiles L_II and N_IJ = inv(L_II) L_IJ; rebuild L_IJ = L_II N_IJ
    std::vector<double> tmp(TT);
    for (int32_t I = 0; I < B.nt; ++I) {
      const TileRow &R = ctx->htrow[B.trow0 + I];
      const double *dI = buf.data() + (R.off - first.off) + (int64_t)(I - R.j0) * TT;
      for (int32_t J = R.j0; J <= I; ++J) {
        const double *t = buf.data() + (R.off - first.off) + (int64_t)(J - R.j0) * TT;
        if (J < I) {
          for (int rr = 0; rr < kTile; ++rr)
            for (int cc = 0; cc < kTile; ++cc) {
              double acc = 0.0;
              for (int kk = 0; kk <= rr; ++kk) acc += dI[rr * kTile + kk] * t[kk * kTile + cc];
              tmp[rr * kTile + cc] = acc;
            }
          t = tmp.data();
        }
        for (int rr = 0; rr < kTile; ++rr) {
          int gr = I * kTile + rr;
          if (gr >= m) break;
          for (int cc = 0; cc < kTile; ++cc) {
            int gc = J * kTile + cc;
            if (gc >= m || gc > gr) break;
            L[(int64_t)gr * m + gc] = t[rr * kTile + cc];
          }
        }
      }
    }
    if (is_fp64) *is_fp64 = B.prec64;
    return CIMMINO_OK;
  } catch (const Error &e) {
    return set_error(ctx, e);
  }
}

// [nrhs][N] (host or device) <-> [N][nrhs] device layout of the CG vectors
static void cols_in(cimmino_ctx *c, const double *V, int32_t nrhs, double *dst, cudaStream_t s) {
  const int64_t N = c->N;
  if (nrhs == 1) {
    h2d(dst, V, N, s);
    return;
  }
  h2d(c->Fin.p, V, N * nrhs, s);
  const int64_t tot = N * nrhs;
  k_cols_to_interleaved<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(c->Fin.p, N, nrhs, dst);
}
static void cols_out(cimmino_ctx *c, const double *src, int32_t nrhs, double *V, cudaStream_t s) {
  const int64_t N = c->N;
  if (nrhs == 1) {
    d2h(V, src, N, s);
    return;
  }
  const int64_t tot = N * nrhs;
  k_interleave_to_cols<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, N, nrhs, c->Fin.p);
  d2h(V, c->Fin.p, N * nrhs, s);
}

int cimmino_project(cimmino_ctx *ctx, const double *v, int32_t nrhs, double *psi,
                    int32_t on_device) {
  if (!ctx || !v || !psi) return CIMMINO_EINVAL;
  try {
    if (ctx->nsys != 1) fail(CIMMINO_EINVAL, "cimmino_project needs a single-system context");
    if (nrhs < 1) fail(CIMMINO_EINVAL, "nrhs must be >= 1");
    (void)on_device;
    ensure_solve_buffers(ctx, nrhs);
    cudaStream_t s = ctx->stream;
    CUDA_TRY(cudaMemsetAsync(ctx->refine_total.p, 0, sizeof(int64_t), s));
    CUDA_TRY(cudaMemsetAsync(ctx->refine_max.p, 0, sizeof(int32_t), s));
    cols_in(ctx, v, nrhs, ctx->p.p, s);
    launch_spmv_plain(ctx->args, ctx->p.p, ctx->u.p, s);
    launch_proj(ctx->args, ctx->u.p, ctx->y.p, 0, s);
    launch_spmv_t(ctx->args, ctx->y.p, ctx->psi.p, s);
    cols_out(ctx, ctx->psi.p, nrhs, psi, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    return CIMMINO_OK;
  } catch (const Error &e) {
    return set_error(ctx, e);
  }
}

int cimmino_project_rhs(cimmino_ctx *ctx, const double *f, int32_t nrhs, double *xi,
                        int32_t on_device) {
  if (!ctx || !f || !xi) return CIMMINO_EINVAL;
  try {
    if (ctx->nsys != 1) fail(CIMMINO_EINVAL, "cimmino_project_rhs needs a single-system context");
    if (nrhs < 1) fail(CIMMINO_EINVAL, "nrhs must be >= 1");
    (void)on_device;
    ensure_solve_buffers(ctx, nrhs);
    cudaStream_t s = ctx->stream;
    CUDA_TRY(cudaMemsetAsync(ctx->cnt.p, 0, sizeof(int32_t) * 4 * ctx->nsys, s));
    h2d(ctx->Fin.p, f, ctx->N * nrhs, s);
    launch_rhs_scale(ctx->args, ctx->Fin.p, ctx->perm.p, s);
    launch_proj(ctx->args, ctx->fs.p, ctx->y.p, 0, s);
    launch_spmv_t(ctx->args, ctx->y.p, ctx->psi.p, s);
    cols_out(ctx, ctx->psi.p, nrhs, xi, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    return CIMMINO_OK;
  } catch (const Error &e) {
    return set_error(ctx, e);
  }
}

int cimmino_sweeps(cimmino_ctx *ctx, const double *f, int32_t nrhs, double omega,
                   int32_t sweeps, double *x, int32_t on_device) {
  if (!ctx || !f || !x) return CIMMINO_EINVAL;
  try {
    if (ctx->nsys != 1) fail(CIMMINO_EINVAL, "cimmino_sweeps needs a single-system context");
    if (nrhs < 1 || sweeps < 0) fail(CIMMINO_EINVAL, "nrhs must be >= 1 and sweeps >= 0");
    if (!std::isfinite(omega)) fail(CIMMINO_EINVAL, "omega must be finite");
    (void)on_device;
    ensure_solve_buffers(ctx, nrhs);
    cudaStream_t s = ctx->stream;
    const int64_t N = ctx->N;
    CUDA_TRY(cudaMemsetAsync(ctx->cnt.p, 0, sizeof(int32_t) * 4 * ctx->nsys, s));
    CUDA_TRY(cudaMemsetAsync(ctx->refine_total.p, 0, sizeof(int64_t), s));
    CUDA_TRY(cudaMemsetAsync(ctx->refine_max.p, 0, sizeof(int32_t), s));
    CUDA_TRY(cudaMemsetAsync(ctx->x.p, 0, sizeof(double) * N * nrhs, s));
    h2d(ctx->Fin.p, f, N * nrhs, s);
    launch_rhs_scale(ctx->args, ctx->Fin.p, ctx->perm.p, s);
    for (int32_t t = 0; t < sweeps; ++t) launch_cim_sweep(ctx->args, omega, s);
    if (ctx->args.cs) launch_unscale_cols(ctx->x.p, ctx->args.cs, N, nrhs, s);
    cols_out(ctx, ctx->x.p, nrhs, x, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    return CIMMINO_OK;
  } catch (const Error &e) {
    return set_error(ctx, e);
  }
}

int cimmino_time_kernels(cimmino_ctx *ctx, int32_t reps, double *ms) {
  if (!ctx || !ms || reps < 1) return CIMMINO_EINVAL;
  try {
    if (ctx->nsys != 1 || ctx->nrhs < 1) fail(CIMMINO_EINVAL, "no solve on this context yet");
    cudaStream_t s = ctx->stream;
    const IterArgs &a = ctx->args;
    Timer t;
    t.start(s);
    for (int32_t i = 0; i < reps; ++i) launch_proj(a, a.u, a.y, 0, s);
    ms[0] = t.stop_ms(s) / reps;
    t.start(s);
    for (int32_t i = 0; i < reps; ++i) launch_spmv_plain(a, a.p, a.u, s);
    ms[1] = t.stop_ms(s) / reps;
    t.start(s);
    for (int32_t i = 0; i < reps; ++i) launch_spmv_t(a, a.y, a.psi, s);
    ms[2] = t.stop_ms(s) / reps;
    CUDA_TRY(cudaGetLastError());
    return CIMMINO_OK;
  } catch (const Error &e) {
    return set_error(ctx, e);
  }
}

int cimmino_aat(const cimmino_csr *A, void *stream, int64_t *nnz, int64_t *row_ptr,
                int32_t *col_idx, double *val) {
  if (!A || !nnz || !row_ptr) {
    g_last_error = "invalid argument";
    return CIMMINO_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    const int64_t N = A->n, NNZ = A->nnz;
    if (N <= 0 || NNZ < 0 || !A->row_ptr || !A->col_idx || (NNZ > 0 && !A->val))
      fail(CIMMINO_EINVAL, "bad CSR header");
    Allocator mem;  // the library pool, ordered on the caller's stream
    mem.stream = s;
    AllocScope scope(&mem);
    DBuf<int64_t> rp, cp, work, tmp, cnt, crp;
    DBuf<int32_t> ci, ri, ovf, flag, cci;
    DBuf<double> va, cv, ccv;
    rp.alloc(N + 1);
    ci.alloc(NNZ);
    va.alloc(NNZ);
    h2d(rp.p, A->row_ptr, N + 1, s);
    h2d(ci.p, A->col_idx, NNZ, s);
    h2d(va.p, A->val, NNZ, s);
    flag.alloc(2);
    CUDA_TRY(cudaMemsetAsync(flag.p, 0, 2 * sizeof(int32_t), s));
    launch_validate_csr(rp.p, ci.p, N, NNZ, flag.p, s);
    int32_t hf = 0;
    d2h(&hf, flag.p, 1, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hf) fail(CIMMINO_EINVAL, "malformed CSR");
    const int64_t tl = scan_tmp_len(N);
    cp.alloc(N + 1);
    ri.alloc(NNZ);
    cv.alloc(NNZ);
    work.alloc(2 * N);
    tmp.alloc(tl);
    launch_transpose(rp.p, ci.p, va.p, N, NNZ, cp.p, ri.p, cv.p, work.p, tmp.p, tl, s);
    cnt.alloc(N);
    ovf.alloc(N + 1);
    spgemm_count(rp.p, ci.p, cp.p, ri.p, N, cnt.p, ovf.p + 1, ovf.p, s);
    int32_t novf = 0;
    d2h(&novf, ovf.p, 1, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    if (novf > 0) {
      spgemm_overflow(rp.p, ci.p, va.p, cp.p, ri.p, ovf.p + 1, novf, cnt.p, nullptr, nullptr,
                      nullptr, flag.p + 1, s);
      d2h(&hf, flag.p + 1, 1, s);
      CUDA_TRY(cudaStreamSynchronize(s));
      if (hf) fail(CIMMINO_EUNSUPPORTED, "a row of A A^T has more than 8192 structural candidates");
    }
    crp.alloc(N + 1);
    launch_scan_counts(cnt.p, crp.p, N, tmp.p, tl, s);
    int64_t nc = 0;
    d2h(&nc, crp.p + N, 1, s);
    CUDA_TRY(cudaStreamSynchronize(s));
    *nnz = nc;
    d2h(row_ptr, crp.p, N + 1, s);
    if (col_idx && val) {
      cci.alloc(nc);
      ccv.alloc(nc);
      spgemm_fill(rp.p, ci.p, va.p, cp.p, ri.p, cv.p, N, crp.p, cci.p, ccv.p, s);
      if (novf > 0)
        spgemm_overflow(rp.p, ci.p, va.p, cp.p, ri.p, ovf.p + 1, novf, cnt.p, crp.p, cci.p,
                        ccv.p, flag.p + 1, s);
      d2h(col_idx, cci.p, nc, s);
      d2h(val, ccv.p, nc, s);
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    return CIMMINO_OK;
  } catch (const Error &e) {
    return set_error(nullptr, e);
  }
}

}  // extern "C"
