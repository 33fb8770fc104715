// Host-side block-row partitioner on the row inner-product graph G_RIP (Section 2.1):
// a vertex per row, an edge (i, j) for every nonzero c_ij = r_i . r_j of C = A A^T,
// with cost |c_ij| / (||r_i|| ||r_j||), i.e. the cosine of the two rows after the unit
// 2-norm prescaling.  A K-way partition minimising the cutsize (Eq. 2.6, the sum of the
// inter-block inner products) under the balance constraint W_k <= cap (Eq. A.1, unit
// vertex weights) is decoded into a row permutation and block offsets (Section 2.2).
//
// This is input plumbing, not the solver's hot path.  Multilevel scheme:
//   coarsen by heavy-edge matching -> recursive bisection of the coarsest graph by
//   greedy graph growing + FM-style refinement -> project back with balance-constrained
//   greedy k-way boundary refinement at every level -> move vertices until every part
//   satisfies the cap.  Inside every part the rows are ordered by reverse Cuthill-McKee
//   on the part's subgraph (the order inside a block row is arbitrary, Section 2.2), which
//   keeps the envelope of the Gram blocks, and hence the skyline factors, small.
//
// Host threads (OpenMP) split the per-vertex work of every phase; the result does not
// depend on the thread count: parallel loops only compute per-vertex proposals from the
// state of the previous round, and every decision that depends on other decisions (which
// matches stand, which moves are applied) is taken in a fixed order.
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include <algorithm>
#include <cmath>
#include <numeric>
#include <queue>
#include <random>
#include <new>
#include <vector>

#include "../../include/cimmino.h"

namespace {

struct Graph {
  int32_t n = 0;
  std::vector<int64_t> xadj;
  std::vector<int32_t> adj;
  std::vector<double> w;
  std::vector<int32_t> vw;
  double total_vw() const {
    double s = 0;
    for (int32_t v : vw) s += v;
    return s;
  }
};

Graph build_rip(int64_t n, const int64_t *crp, const int32_t *cci, const double *ccv) {
  Graph g;
  g.n = (int32_t)n;
  std::vector<double> d(n, 1.0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t q = crp[i]; q < crp[i + 1]; ++q)
      if (cci[q] == i && ccv[q] > 0) d[i] = std::sqrt(ccv[q]);
  g.xadj.assign(n + 1, 0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = 0;
    for (int64_t q = crp[i]; q < crp[i + 1]; ++q)
      if (cci[q] != i && ccv[q] != 0.0) ++c;
    g.xadj[i + 1] = c;
  }
  for (int64_t i = 0; i < n; ++i) g.xadj[i + 1] += g.xadj[i];
  g.adj.resize(g.xadj[n]);
  g.w.resize(g.xadj[n]);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t o = g.xadj[i];
    for (int64_t q = crp[i]; q < crp[i + 1]; ++q)
      if (cci[q] != i && ccv[q] != 0.0) {
        g.adj[o] = cci[q];
        g.w[o] = std::fabs(ccv[q]) / (d[i] * d[cci[q]]);
        ++o;
      }
  }
  g.vw.assign(n, 1);
  return g;
}

// Tie-break of equal edge weights in the matching: a hash of the (unordered) edge and the
// level's seed, so that the choice is random-like but the same for both end points.
inline uint64_t edge_hash(uint64_t a, uint64_t b, uint64_t seed) {
  if (a > b) std::swap(a, b);
  uint64_t x = (a * 0x9E3779B97F4A7C15ull) ^ (b + 0x632BE59BD9B4E019ull) ^ seed;
  x ^= x >> 31;
  x *= 0xBF58476D1CE4E5B9ull;
  x ^= x >> 29;
  return x;
}

// Heavy-edge matching by rounds of mutual proposals: every unmatched vertex proposes to its
// heaviest unmatched neighbour that keeps the coarse weight under maxvw (ties broken by the
// edge hash); mutual proposals are matched.  cmap[v] = coarse vertex of v.
Graph coarsen(const Graph &g, int32_t maxvw, uint64_t seed, std::vector<int32_t> &cmap) {
  const int32_t n = g.n;
  std::vector<int32_t> match(n, -1), prop(n, -1);
  for (int round = 0; round < 6; ++round) {
    int64_t open = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : open)
    for (int32_t v = 0; v < n; ++v) {
      prop[v] = -1;
      if (match[v] != -1) continue;
      int32_t best = -1;
      double bw = -1.0;
      uint64_t bh = 0;
      for (int64_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) {
        const int32_t u = g.adj[q];
        if (g.w[q] < bw || match[u] != -1 || u == v || g.vw[u] + g.vw[v] > maxvw) continue;
        if (g.w[q] > bw) {
          bw = g.w[q];
          bh = edge_hash((uint64_t)u, (uint64_t)v, seed);
          best = u;
        } else {  // equal weights: the edge hash decides
          const uint64_t h = edge_hash((uint64_t)u, (uint64_t)v, seed);
          if (h > bh) {
            bh = h;
            best = u;
          }
        }
      }
      prop[v] = best;
      open += best >= 0;
    }
    if (!open) break;
#pragma omp parallel for schedule(static)
    for (int32_t v = 0; v < n; ++v) {
      const int32_t u = prop[v];
      if (u >= 0 && prop[u] == v) match[v] = u;  // both ends write the same pair
    }
  }
  cmap.assign(n, -1);
  int32_t nc = 0;
  std::vector<int32_t> rep;
  rep.reserve(n / 2 + 1);
  for (int32_t v = 0; v < n; ++v) {
    if (match[v] == -1) match[v] = v;
    if (cmap[v] == -1) {
      cmap[v] = nc;
      cmap[match[v]] = nc;
      rep.push_back(v);
      ++nc;
    }
  }
  Graph c;
  c.n = nc;
  c.vw.assign(nc, 0);
#pragma omp parallel for schedule(static)
  for (int32_t cv = 0; cv < nc; ++cv) {
    const int32_t a = rep[cv], b = match[a];
    c.vw[cv] = g.vw[a] + (b != a ? g.vw[b] : 0);
  }
  // coarse adjacency: chunks of coarse vertices in parallel into per-chunk buffers (the
  // edge order of a coarse vertex is that of the sequential program), then concatenated
  constexpr int32_t kChunk = 8192;
  const int32_t nchunk = (nc + kChunk - 1) / kChunk;
  std::vector<std::vector<int32_t>> cadj(nchunk);
  std::vector<std::vector<double>> cw(nchunk);
  std::vector<int64_t> deg(nc, 0);
#pragma omp parallel
  {
    std::vector<int32_t> mark(nc, -1), list;
    std::vector<double> acc(nc, 0.0);
#pragma omp for schedule(dynamic, 1)
    for (int32_t ch = 0; ch < nchunk; ++ch) {
      const int32_t c0 = ch * kChunk, c1 = std::min(nc, c0 + kChunk);
      for (int32_t cv = c0; cv < c1; ++cv) {
        list.clear();
        const int32_t a = rep[cv], b = match[a];
        auto gather = [&](int32_t v) {
          for (int64_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) {
            const int32_t cu = cmap[g.adj[q]];
            if (cu == cv) continue;
            if (mark[cu] != cv) {
              mark[cu] = cv;
              acc[cu] = 0.0;
              list.push_back(cu);
            }
            acc[cu] += g.w[q];
          }
        };
        gather(a);
        if (b != a) gather(b);  // an unmatched vertex (b == a) has no partner
        for (int32_t cu : list) {
          cadj[ch].push_back(cu);
          cw[ch].push_back(acc[cu]);
        }
        deg[cv] = (int64_t)list.size();
      }
    }
  }
  c.xadj.assign(nc + 1, 0);
  for (int32_t cv = 0; cv < nc; ++cv) c.xadj[cv + 1] = c.xadj[cv] + deg[cv];
  c.adj.resize(c.xadj[nc]);
  c.w.resize(c.xadj[nc]);
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t ch = 0; ch < nchunk; ++ch) {
    const int64_t o = c.xadj[(int64_t)ch * kChunk];
    std::copy(cadj[ch].begin(), cadj[ch].end(), c.adj.begin() + o);
    std::copy(cw[ch].begin(), cw[ch].end(), c.w.begin() + o);
  }
  return c;
}

// cut of a partition
double cut_of(const Graph &g, const std::vector<int32_t> &part) {
  double s = 0;
  for (int32_t v = 0; v < g.n; ++v)
    for (int64_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q)
      if (g.adj[q] > v && part[g.adj[q]] != part[v]) s += g.w[q];
  return s;
}

// Bisect the vertex subset `vs` (part ids p0 / p1) so that side 0 weighs about target0:
// greedy growing from a pseudo-peripheral vertex, then FM-style passes of single moves.
void bisect(const Graph &g, const std::vector<int32_t> &vs, double target0, int32_t p0, int32_t p1,
            std::vector<int32_t> &part, std::mt19937_64 &rng) {
  if (vs.empty()) return;
  std::vector<int32_t> local(g.n, -1);
  for (size_t i = 0; i < vs.size(); ++i) local[vs[i]] = (int32_t)i;
  const size_t m = vs.size();
  // pseudo-peripheral seed: farthest vertex (BFS) from a random start, twice
  auto bfs_far = [&](int32_t s) {
    std::vector<int32_t> dist(m, -1), q;
    q.push_back(s);
    dist[local[s]] = 0;
    int32_t last = s;
    for (size_t h = 0; h < q.size(); ++h) {
      const int32_t v = q[h];
      last = v;
      for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
        const int32_t u = g.adj[e];
        if (local[u] >= 0 && dist[local[u]] < 0) {
          dist[local[u]] = dist[local[v]] + 1;
          q.push_back(u);
        }
      }
    }
    return last;
  };
  int32_t seed = vs[rng() % m];
  seed = bfs_far(bfs_far(seed));
  // greedy growing: add the frontier vertex with the largest gain 2 conn - tot, where conn
  // is its edge weight into the grown region and tot its edge weight inside vs; a lazy
  // max-heap holds (gain, vertex) entries, stale ones are skipped when popped
  std::vector<char> in(m, 0);
  std::vector<double> conn(m, 0.0), tot(m, 0.0);
  for (size_t i = 0; i < m; ++i)
    for (int64_t e = g.xadj[vs[i]]; e < g.xadj[vs[i] + 1]; ++e)
      if (local[g.adj[e]] >= 0) tot[i] += g.w[e];
  std::priority_queue<std::pair<double, int32_t>> heap;
  double wgrown = 0;
  auto add = [&](int32_t li) {
    in[li] = 1;
    wgrown += g.vw[vs[li]];
    for (int64_t e = g.xadj[vs[li]]; e < g.xadj[vs[li] + 1]; ++e) {
      const int32_t lu = local[g.adj[e]];
      if (lu >= 0 && !in[lu]) {
        conn[lu] += g.w[e];
        heap.emplace(2 * conn[lu] - tot[lu], lu);
      }
    }
  };
  add(local[seed]);
  size_t next_unvisited = 0;
  while (wgrown < target0) {
    int32_t best = -1;
    while (!heap.empty()) {
      const auto top = heap.top();
      heap.pop();
      if (!in[top.second] && top.first == 2 * conn[top.second] - tot[top.second]) {
        best = top.second;
        break;
      }
    }
    if (best < 0) {  // disconnected remainder: restart from any vertex not yet grown
      while (next_unvisited < m && in[next_unvisited]) ++next_unvisited;
      if (next_unvisited >= m) break;
      best = (int32_t)next_unvisited;
    }
    const int32_t vwb = g.vw[vs[best]];
    if (wgrown + vwb > target0 + 0.5 * vwb && wgrown > 0) break;
    add(best);
  }
  for (size_t i = 0; i < m; ++i) part[vs[i]] = in[i] ? p0 : p1;
  // FM-style refinement: single moves with positive gain that keep the balance within 2%
  double w0 = 0, wtot = 0;
  for (int32_t v : vs) {
    wtot += g.vw[v];
    if (part[v] == p0) w0 += g.vw[v];
  }
  const double tol = std::max(2.0, 0.02 * wtot);
  for (int pass = 0; pass < 6; ++pass) {
    int moved = 0;
    for (int32_t v : vs) {
      double ext = 0, intw = 0;
      for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
        const int32_t u = g.adj[e];
        if (local[u] < 0) continue;
        (part[u] == part[v] ? intw : ext) += g.w[e];
      }
      if (ext <= intw) continue;
      const bool to1 = part[v] == p0;
      const double nw0 = w0 + (to1 ? -g.vw[v] : g.vw[v]);
      if (std::fabs(nw0 - target0) > tol && std::fabs(nw0 - target0) >= std::fabs(w0 - target0))
        continue;
      part[v] = to1 ? p1 : p0;
      w0 = nw0;
      ++moved;
    }
    if (!moved) break;
  }
}

// Parts k0 .. k0 + K - 1 of the vertex subset vs.  The two halves touch disjoint vertices
// and draw from generators of their own (seeded by the part range), so they run as
// independent tasks and the result does not depend on the schedule.
void recursive_bisection(const Graph &g, const std::vector<int32_t> &vs, int32_t k0, int32_t K,
                         std::vector<int32_t> &part, uint64_t seed) {
  if (K <= 1 || vs.empty()) {
    for (int32_t v : vs) part[v] = k0;
    return;
  }
  const int32_t K1 = K / 2;
  double w = 0;
  for (int32_t v : vs) w += g.vw[v];
  std::mt19937_64 rng(seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(k0 + 1)) ^ (uint64_t)K << 40);
  bisect(g, vs, w * K1 / K, k0, k0 + K1, part, rng);
  std::vector<int32_t> a, b;
  for (int32_t v : vs) (part[v] == k0 ? a : b).push_back(v);
#pragma omp task shared(g, part) firstprivate(a) if (a.size() > 4096)
  recursive_bisection(g, a, k0, K1, part, seed);
#pragma omp task shared(g, part) firstprivate(b) if (b.size() > 4096)
  recursive_bisection(g, b, k0 + K1, K - K1, part, seed);
#pragma omp taskwait
}

// Balance-constrained greedy k-way refinement of the boundary.  Each pass: every vertex
// proposes its best move (largest gain in edge weight kept inside its part) from the current
// assignment, in parallel; then the proposals are applied in vertex order, each after its
// gain is recomputed against the assignment as it stands and the cap is checked.
void refine_kway(const Graph &g, std::vector<int32_t> &part, int32_t K, double cap,
                 int passes) {
  std::vector<double> size(K, 0.0);
  for (int32_t v = 0; v < g.n; ++v) size[part[v]] += g.vw[v];
  std::vector<int32_t> prop(g.n, -1);
  auto best_move = [&](int32_t v, std::vector<double> &conn, std::vector<int32_t> &touched,
                       bool check_cap, double &gain) {
    const int32_t pv = part[v];
    touched.clear();
    bool boundary = false;
    for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
      const int32_t p = part[g.adj[e]];
      if (conn[p] == 0.0) touched.push_back(p);
      conn[p] += g.w[e];
      boundary |= p != pv;
    }
    int32_t best = -1;
    double bgain = 0.0;
    if (boundary)
      for (int32_t p : touched) {
        if (p == pv || (check_cap && size[p] + g.vw[v] > cap)) continue;
        const double gn = conn[p] - conn[pv];
        if (gn > bgain || (gn == bgain && best >= 0 && p < best)) {
          bgain = gn;
          best = p;
        }
      }
    for (int32_t p : touched) conn[p] = 0.0;
    gain = bgain;
    return best;
  };
  std::vector<double> conn(K, 0.0);
  std::vector<int32_t> touched;
  for (int pass = 0; pass < passes; ++pass) {
#pragma omp parallel
    {
      std::vector<double> lconn(K, 0.0);
      std::vector<int32_t> ltouched;
      double gn;
#pragma omp for schedule(dynamic, 4096)
      for (int32_t v = 0; v < g.n; ++v) prop[v] = best_move(v, lconn, ltouched, true, gn);
    }
    int64_t moved = 0;
    for (int32_t v = 0; v < g.n; ++v) {
      if (prop[v] < 0) continue;
      double gn;
      const int32_t best = best_move(v, conn, touched, true, gn);
      if (best < 0) continue;
      const int32_t pv = part[v];
      part[v] = best;
      size[pv] -= g.vw[v];
      size[best] += g.vw[v];
      ++moved;
    }
    if (moved <= g.n / 2000) break;  // converged: further passes gain little
  }
}

// Move vertices out of parts above the cap.  Every round collects, for each vertex of an
// over-full part, its best move into an under-full part it touches (loss = edge weight it
// keeps minus edge weight it gains), then applies the moves cheapest first while both
// parts still need them.  A part with no such neighbour sends vertices to the lightest part.
void enforce_cap(const Graph &g, std::vector<int32_t> &part, int32_t K, int32_t cap) {
  std::vector<int64_t> size(K, 0);
  for (int32_t v = 0; v < g.n; ++v) size[part[v]] += 1;
  struct Move {
    double loss;
    int32_t v, to;
  };
  std::vector<Move> cand;
  for (int round = 0; round < 16; ++round) {
    bool over = false;
    for (int32_t k = 0; k < K; ++k) over |= size[k] > cap;
    if (!over) return;
    cand.clear();
    std::vector<int32_t> to(g.n, -1);
    std::vector<double> loss(g.n, 0.0);
#pragma omp parallel
    {
      std::vector<double> lconn(K, 0.0);
      std::vector<int32_t> ltouched;
#pragma omp for schedule(dynamic, 4096)
      for (int32_t v = 0; v < g.n; ++v) {
        const int32_t pv = part[v];
        if (size[pv] <= cap) continue;
        ltouched.clear();
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
          const int32_t p = part[g.adj[e]];
          if (lconn[p] == 0.0) ltouched.push_back(p);
          lconn[p] += g.w[e];
        }
        int32_t best = -1;
        double bl = 1e300;
        for (int32_t p : ltouched)
          if (p != pv && size[p] < cap &&
              (lconn[pv] - lconn[p] < bl || (lconn[pv] - lconn[p] == bl && p < best))) {
            bl = lconn[pv] - lconn[p];
            best = p;
          }
        to[v] = best;
        loss[v] = bl;
        for (int32_t p : ltouched) lconn[p] = 0.0;
      }
    }
    for (int32_t v = 0; v < g.n; ++v)
      if (to[v] >= 0) cand.push_back({loss[v], v, to[v]});
    if (cand.empty()) break;
    std::stable_sort(cand.begin(), cand.end(),
                     [](const Move &a, const Move &b) { return a.loss < b.loss; });
    int64_t moved = 0;
    for (const Move &m : cand) {
      const int32_t pv = part[m.v];
      if (size[pv] <= cap || size[m.to] >= cap) continue;
      part[m.v] = m.to;
      --size[pv];
      ++size[m.to];
      ++moved;
    }
    if (!moved) break;
  }
  // last resort: fill the lightest parts
  for (int32_t v = 0; v < g.n; ++v) {
    const int32_t pv = part[v];
    if (size[pv] <= cap) continue;
    int32_t lo = (int32_t)(std::min_element(size.begin(), size.end()) - size.begin());
    part[v] = lo;
    --size[pv];
    ++size[lo];
  }
}

// reverse Cuthill-McKee order of the vertices of one part (on its induced subgraph)
void rcm_order(const Graph &g, const std::vector<int32_t> &vs, std::vector<int32_t> &out,
               std::vector<int32_t> &local) {
  const size_t m = vs.size();
  for (size_t i = 0; i < m; ++i) local[vs[i]] = (int32_t)i;
  std::vector<int32_t> deg(m, 0);
  for (size_t i = 0; i < m; ++i)
    for (int64_t e = g.xadj[vs[i]]; e < g.xadj[vs[i] + 1]; ++e) deg[i] += local[g.adj[e]] >= 0;
  std::vector<char> seen(m, 0);
  std::vector<int32_t> order;
  order.reserve(m);
  std::vector<int32_t> nb;
  for (size_t start = 0; order.size() < m;) {
    // start of the next component: unseen vertex of minimum degree, then a BFS-far vertex
    int32_t s = -1;
    for (size_t i = 0; i < m; ++i)
      if (!seen[i] && (s < 0 || deg[i] < deg[s])) s = (int32_t)i;
    auto bfs = [&](int32_t root, bool commit) {
      std::vector<int32_t> q{root};
      std::vector<char> vis(m, 0);
      vis[root] = 1;
      for (size_t h = 0; h < q.size(); ++h) {
        const int32_t v = q[h];
        nb.clear();
        for (int64_t e = g.xadj[vs[v]]; e < g.xadj[vs[v] + 1]; ++e) {
          const int32_t u = local[g.adj[e]];
          if (u >= 0 && !vis[u] && !seen[u]) {
            vis[u] = 1;
            nb.push_back(u);
          }
        }
        std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
          return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
        });
        q.insert(q.end(), nb.begin(), nb.end());
      }
      if (commit)
        for (int32_t v : q) {
          seen[v] = 1;
          order.push_back(v);
        }
      return q.back();
    };
    const int32_t far = bfs(s, false);
    bfs(far, true);
    (void)start;
  }
  out.clear();
  for (size_t i = m; i-- > 0;) out.push_back(vs[order[i]]);
  for (size_t i = 0; i < m; ++i) local[vs[i]] = -1;
}

}  // namespace

extern "C" int cimmino_partition_rip(int64_t n, const int64_t *crp, const int32_t *cci,
                                     const double *ccv, int32_t K, int32_t cap, uint64_t seed,
                                     int32_t *perm, int64_t *block_ptr, double *cutsize) {
  if (n <= 0 || !crp || !cci || !ccv || !perm || !block_ptr || K < 1 || K > n ||
      (int64_t)cap * K < n)
    return CIMMINO_EINVAL;
  try {
    std::vector<Graph> levels;
    std::vector<std::vector<int32_t>> maps;
    levels.push_back(build_rip(n, crp, cci, ccv));
    // coarsen until a few dozen vertices per part remain
    const int32_t maxvw = std::max(1, cap / 32);
    while (levels.back().n > std::max<int64_t>(40LL * K, 2000)) {
      std::vector<int32_t> cmap;
      Graph c = coarsen(levels.back(), maxvw, seed + 0x51ED2700ull * levels.size(), cmap);
      if (c.n > 0.92 * levels.back().n) break;
      maps.push_back(std::move(cmap));
      levels.push_back(std::move(c));
    }
    // initial partition of the coarsest graph
    const Graph &gc = levels.back();
    std::vector<int32_t> part(gc.n, 0), all(gc.n);
    std::iota(all.begin(), all.end(), 0);
#pragma omp parallel
#pragma omp single
    recursive_bisection(gc, all, 0, K, part, seed);
    // uncoarsen with refinement; the cap loosens toward the coarse levels
    for (int lvl = (int)levels.size() - 1; lvl >= 0; --lvl) {
      const Graph &g = levels[lvl];
      const double slack = lvl == 0 ? 1.0 : 1.0 + 0.03 * lvl;
      refine_kway(g, part, K, cap * slack, 8);
      if (lvl > 0) {
        std::vector<int32_t> fine(levels[lvl - 1].n);
        for (int32_t v = 0; v < levels[lvl - 1].n; ++v) fine[v] = part[maps[lvl - 1][v]];
        part.swap(fine);
      }
    }
    const Graph &g = levels.front();
    enforce_cap(g, part, K, cap);
    refine_kway(g, part, K, cap, 4);
    // every part must hold at least one row: borrow from the largest parts
    std::vector<int64_t> size(K, 0);
    for (int64_t v = 0; v < n; ++v) ++size[part[v]];
    for (int32_t k = 0; k < K; ++k)
      while (size[k] == 0) {
        const int32_t big = (int32_t)(std::max_element(size.begin(), size.end()) - size.begin());
        for (int64_t v = 0; v < n; ++v)
          if (part[v] == big) {
            part[v] = k;
            --size[big];
            ++size[k];
            break;
          }
      }
    if (cutsize) *cutsize = cut_of(g, part);
    // decode: parts in order, RCM inside each part
    std::vector<std::vector<int32_t>> members(K);
    for (int64_t v = 0; v < n; ++v) members[part[v]].push_back((int32_t)v);
    block_ptr[0] = 0;
    for (int32_t k = 0; k < K; ++k) block_ptr[k + 1] = block_ptr[k] + (int64_t)members[k].size();
    // parts are ordered independently (a local index array per thread)
#pragma omp parallel
    {
      std::vector<int32_t> local(n, -1), ord;
#pragma omp for schedule(dynamic, 1)
      for (int32_t k = 0; k < K; ++k) {
        rcm_order(g, members[k], ord, local);
        std::copy(ord.begin(), ord.end(), perm + block_ptr[k]);
      }
    }
    return CIMMINO_OK;
  } catch (...) {
    return CIMMINO_ENOMEM;
  }
}

// Section 2.3, dense columns: a column of A with more than sqrt(n) nonzeros makes the
// rows that share it pairwise adjacent, so C = A A^T, and the graph, turn dense.  The
// graph is therefore built from a copy of A in which every column with more than
// t = floor(sqrt(n)) nonzeros keeps only its t entries of largest magnitude; equal
// magnitudes keep the lower row first, so the kept set is unique.  The solve itself
// always uses the full A.
extern "C" int cimmino_sparsify_dense_columns(int64_t n, const int64_t *rp, const int32_t *ci,
                                              const double *val, int64_t *out_rp,
                                              int32_t *out_ci, double *out_val,
                                              int64_t *nnz_out) {
  if (n < 1 || !rp || !ci || !val || !out_rp || !out_ci || !out_val || !nnz_out)
    return CIMMINO_EINVAL;
  const int64_t nnz = rp[n];
  if (rp[0] != 0 || nnz < 0) return CIMMINO_EINVAL;
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return CIMMINO_EINVAL;
  int64_t t = (int64_t)std::sqrt((double)n);
  while (t * t > n) --t;
  while ((t + 1) * (t + 1) <= n) ++t;
  try {
    std::vector<int64_t> cnt(n + 1, 0);
    for (int64_t q = 0; q < nnz; ++q) {
      if (ci[q] < 0 || ci[q] >= n) return CIMMINO_EINVAL;
      ++cnt[ci[q] + 1];
    }
    std::vector<char> keep(nnz, 1);
    // entries of the dense columns, grouped by column (rows increasing inside a column)
    std::vector<int64_t> start(n + 1, 0);
    for (int64_t j = 0; j < n; ++j) start[j + 1] = start[j] + (cnt[j + 1] > t ? cnt[j + 1] : 0);
    if (start[n] > 0) {
      std::vector<int64_t> pos(start[n]);
      std::vector<int32_t> row(start[n]);
      std::vector<int64_t> fill(start.begin(), start.end() - 1);
      for (int64_t i = 0; i < n; ++i)
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
          if (cnt[ci[q] + 1] > t) {
            const int64_t w = fill[ci[q]]++;
            pos[w] = q;
            row[w] = (int32_t)i;
          }
      std::vector<int64_t> idx;
      for (int64_t j = 0; j < n; ++j) {
        const int64_t a = start[j], b = start[j + 1];
        if (b == a) continue;
        idx.resize(b - a);
        std::iota(idx.begin(), idx.end(), a);
        auto before = [&](int64_t x, int64_t y) {
          const double ax = std::fabs(val[pos[x]]), ay = std::fabs(val[pos[y]]);
          return ax > ay || (ax == ay && row[x] < row[y]);
        };
        std::nth_element(idx.begin(), idx.begin() + t, idx.end(), before);
        for (size_t k = (size_t)t; k < idx.size(); ++k) keep[pos[idx[k]]] = 0;
      }
    }
    int64_t w = 0;
    out_rp[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
        if (keep[q]) {
          out_ci[w] = ci[q];
          out_val[w] = val[q];
          ++w;
        }
      out_rp[i + 1] = w;
    }
    *nnz_out = w;
  } catch (const std::bad_alloc &) {
    return CIMMINO_ENOMEM;
  }
  return CIMMINO_OK;
}
