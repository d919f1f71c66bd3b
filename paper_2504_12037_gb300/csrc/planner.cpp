// Width-set finder (Sec. 2): choose the spins W whose configurations are
// enumerated (sampled by the MADE) so that the rest of the network, R, can be
// contracted exactly with every intermediate factor over at most w_u spins.
//
// Width of an elimination: eliminating spin v from the graph on R (with the
// fill edges of the earlier eliminations) produces a factor over v's current
// neighbours; the width of an order is the largest such neighbour count.
// w_u = 1 leaves a forest (W is a feedback vertex set); the GPU elimination
// kernels take widths up to 12.
//
// Two searches, each restarted with different random tie-breaks:
//  * fixed order (the paper's route): a min-fill order of the whole graph,
//    then dynamic slicing along it -- repeatedly move into W the spin that
//    occurs in the most factors of maximum width, until the width is at most
//    w_u -- then return sliced spins to R one at a time, in random order,
//    whenever the width stays within w_u;
//  * greedy: build the order and the slicing together -- eliminate a spin of
//    degree <= w_u (least fill first) while there is one, otherwise slice the
//    spin of largest degree -- then the same return step, each trial checked
//    by a fresh greedy elimination without slicing.
// The smaller W over all trials wins.  Optionally the winner is then
// annealed (the paper also anneals): a random sliced spin returns to R, a
// greedy elimination with slicing repairs the width (possibly slicing
// others), and the move is accepted by the Metropolis rule on |W| under a
// linearly falling temperature; the smallest set seen is kept.  Host code
// only: no device work.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/tnvan.h"

namespace {

struct Rng {  // splitmix64
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
  }
  int below(int n) { return (int)(next() % (uint64_t)n); }
};

// Symmetric adjacency as one bitset row per spin.
struct Graph {
  int n = 0, words = 0;
  std::vector<uint64_t> bits;
  uint64_t* row(int v) { return bits.data() + (size_t)v * words; }
  const uint64_t* row(int v) const { return bits.data() + (size_t)v * words; }
  bool has(int a, int b) const { return (row(a)[b >> 6] >> (b & 63)) & 1; }
  void set(int a, int b) { row(a)[b >> 6] |= 1ull << (b & 63); }
  void clear(int a, int b) { row(a)[b >> 6] &= ~(1ull << (b & 63)); }
};

template <class F>
inline void for_each_bit(const uint64_t* r, int words, F f) {
  for (int k = 0; k < words; ++k) {
    uint64_t x = r[k];
    while (x) {
      const int b = __builtin_ctzll(x);
      f(k * 64 + b);
      x &= x - 1;
    }
  }
}

inline int popcount_row(const uint64_t* r, int words) {
  int c = 0;
  for (int k = 0; k < words; ++k) c += __builtin_popcountll(r[k]);
  return c;
}

// Elimination state on the spins not removed: the filled graph, degrees and
// cached fill counts (pairs of neighbours not yet adjacent).
struct Elim {
  Graph g;
  std::vector<char> alive;
  std::vector<int> deg, fill;
  std::vector<char> dirty;
  std::vector<int> nb;  // scratch

  void init(const Graph& base, const std::vector<char>& removed) {
    g = base;
    const int n = g.n;
    alive.assign(n, 1);
    for (int v = 0; v < n; ++v)
      if (removed[v]) drop(v, false);
    deg.assign(n, 0);
    for (int v = 0; v < n; ++v) deg[v] = alive[v] ? popcount_row(g.row(v), g.words) : 0;
    fill.assign(n, 0);
    dirty.assign(n, 1);
  }
  // remove v from the graph without fill (slicing) or after its neighbours
  // were joined (elimination)
  void drop(int v, bool track) {
    alive[v] = 0;
    nb.clear();
    for_each_bit(g.row(v), g.words, [&](int a) { nb.push_back(a); });
    for (int a : nb) {
      g.clear(a, v);
      if (track) --deg[a];
    }
    std::memset(g.row(v), 0, sizeof(uint64_t) * g.words);
    if (track) {
      deg[v] = 0;
      mark_near(nb);
    }
  }
  void mark_near(const std::vector<int>& around) {
    for (int a : around) {
      dirty[a] = 1;
      for_each_bit(g.row(a), g.words, [&](int u) { dirty[u] = 1; });
    }
  }
  int fill_of(int v) {
    if (!dirty[v]) return fill[v];
    std::vector<int> ns;
    for_each_bit(g.row(v), g.words, [&](int a) { ns.push_back(a); });
    int f = 0;
    for (size_t i = 0; i < ns.size(); ++i)
      for (size_t j = i + 1; j < ns.size(); ++j)
        if (!g.has(ns[i], ns[j])) ++f;
    fill[v] = f;
    dirty[v] = 0;
    return f;
  }
  // join v's neighbours pairwise, then remove v; returns the factor width
  int eliminate(int v) {
    std::vector<int> ns;
    for_each_bit(g.row(v), g.words, [&](int a) { ns.push_back(a); });
    for (size_t i = 0; i < ns.size(); ++i)
      for (size_t j = i + 1; j < ns.size(); ++j)
        if (!g.has(ns[i], ns[j])) {
          g.set(ns[i], ns[j]);
          g.set(ns[j], ns[i]);
          ++deg[ns[i]];
          ++deg[ns[j]];
        }
    const int w = (int)ns.size();
    drop(v, true);
    return w;
  }
};

// Uniform choice among ties: reservoir over candidates with equal key.
struct Pick {
  int best = -1;
  long key = 0;
  int ties = 0;
  void offer(int v, long k, Rng* rng, bool lower_better) {
    const bool better = best < 0 || (lower_better ? k < key : k > key);
    if (better) {
      best = v;
      key = k;
      ties = 1;
    } else if (k == key) {
      ++ties;
      if (rng ? rng->below(ties) == 0 : v < best) best = v;
    }
  }
};

// Greedy elimination of the spins not in `removed`; with slice, spins that
// block it are moved into W (appended to slice_out).  Returns false when it
// gets stuck without slicing.  order_out: eliminated spins in order.
bool greedy(const Graph& base, const std::vector<char>& removed, int wu, bool slice, Rng* rng,
            std::vector<int>* order_out, std::vector<int>* slice_out) {
  Elim e;
  e.init(base, removed);
  const int n = base.n;
  int left = 0;
  for (int v = 0; v < n; ++v) left += e.alive[v];
  if (order_out) order_out->clear();
  while (left > 0) {
    Pick p;
    for (int v = 0; v < n; ++v)
      if (e.alive[v] && e.deg[v] <= wu) p.offer(v, e.fill_of(v), rng, true);
    if (p.best >= 0) {
      e.eliminate(p.best);
      if (order_out) order_out->push_back(p.best);
    } else {
      if (!slice) return false;
      Pick q;
      for (int v = 0; v < n; ++v)
        if (e.alive[v]) q.offer(v, e.deg[v], rng, false);
      e.drop(q.best, true);
      slice_out->push_back(q.best);
    }
    --left;
  }
  return true;
}

// Min-fill order of the whole graph (no width limit).
std::vector<int> minfill_order(const Graph& base, Rng* rng) {
  std::vector<char> none(base.n, 0);
  std::vector<int> order;
  greedy(base, none, base.n, false, rng, &order, nullptr);
  return order;
}

// Eliminate along `order` skipping removed spins; returns the width and, when
// counts is given, per spin the number of maximum-width factors it is in
// (the eliminated spin included).
int width_along(const Graph& base, const std::vector<int>& order, const std::vector<char>& removed,
                std::vector<int>* counts) {
  Elim e;
  e.init(base, removed);
  std::vector<int> w(order.size(), -1);
  std::vector<std::vector<int>> scope;
  if (counts) scope.resize(order.size());
  int wmax = 0;
  for (size_t k = 0; k < order.size(); ++k) {
    const int v = order[k];
    if (removed[v]) continue;
    if (counts) for_each_bit(e.g.row(v), e.g.words, [&](int a) { scope[k].push_back(a); });
    w[k] = e.eliminate(v);
    wmax = std::max(wmax, w[k]);
  }
  if (counts) {
    counts->assign(base.n, 0);
    for (size_t k = 0; k < order.size(); ++k)
      if (w[k] == wmax && wmax > 0) {
        ++(*counts)[order[k]];
        for (int a : scope[k]) ++(*counts)[a];
      }
  }
  return wmax;
}

struct Result {
  std::vector<int> W, order;
  int width = 0;
};

Result search_fixed(const Graph& G, int wu, Rng& rng) {
  const int n = G.n;
  Result r;
  r.order = minfill_order(G, &rng);
  std::vector<char> removed(n, 0);
  std::vector<int> counts;
  int w = width_along(G, r.order, removed, &counts);
  while (w > wu) {
    Pick p;
    for (int v = 0; v < n; ++v)
      if (!removed[v] && counts[v] > 0) p.offer(v, counts[v], &rng, false);
    removed[p.best] = 1;
    r.W.push_back(p.best);
    w = width_along(G, r.order, removed, &counts);
  }
  std::vector<int> trial(r.W);
  for (size_t i = trial.size(); i > 1; --i) std::swap(trial[i - 1], trial[rng.below((int)i)]);
  for (int u : trial) {
    removed[u] = 0;
    if (width_along(G, r.order, removed, nullptr) > wu) removed[u] = 1;
  }
  std::vector<int> keep;
  for (int u : r.W)
    if (removed[u]) keep.push_back(u);
  r.W.swap(keep);
  std::vector<int> ord;
  for (int v : r.order)
    if (!removed[v]) ord.push_back(v);
  r.order.swap(ord);
  r.width = width_along(G, r.order, removed, nullptr);
  return r;
}

Result search_greedy(const Graph& G, int wu, Rng& rng) {
  const int n = G.n;
  Result r;
  std::vector<char> removed(n, 0);
  greedy(G, removed, wu, true, &rng, &r.order, &r.W);
  for (int u : r.W) removed[u] = 1;
  std::vector<int> trial(r.W), ord;
  for (size_t i = trial.size(); i > 1; --i) std::swap(trial[i - 1], trial[rng.below((int)i)]);
  for (int u : trial) {
    removed[u] = 0;
    if (greedy(G, removed, wu, false, &rng, &ord, nullptr)) r.order = ord;
    else removed[u] = 1;
  }
  std::vector<int> keep;
  for (int u : r.W)
    if (removed[u]) keep.push_back(u);
  r.W.swap(keep);
  r.width = width_along(G, r.order, removed, nullptr);
  return r;
}

Result search_anneal(const Graph& G, int wu, Rng& rng, const Result& start, int iters, double T0) {
  const int n = G.n;
  std::vector<char> inW(n, 0);
  for (int u : start.W) inW[u] = 1;
  std::vector<int> cur(start.W), ord, extra;
  Result best = start;
  for (int it = 0; it < iters && !cur.empty(); ++it) {
    const double T = T0 * (1.0 - (double)it / iters) + 1e-3;
    const int pick = rng.below((int)cur.size());
    const int u = cur[pick];
    std::vector<char> removed(inW);
    removed[u] = 0;
    extra.clear();
    greedy(G, removed, wu, true, &rng, &ord, &extra);
    const int delta = (int)extra.size() - 1;
    const double accept = delta <= 0 ? 1.0 : std::exp(-delta / T);
    const double r = (double)(rng.next() >> 11) * (1.0 / 9007199254740992.0);
    if (r < accept) {
      inW[u] = 0;
      cur.erase(cur.begin() + pick);
      for (int v : extra) {
        inW[v] = 1;
        cur.push_back(v);
      }
      if (cur.size() < best.W.size()) {
        best.W = cur;
        best.order = ord;
      }
    }
  }
  std::vector<char> removed(n, 0);
  for (int u : best.W) removed[u] = 1;
  best.width = width_along(G, best.order, removed, nullptr);
  return best;
}

}  // namespace

extern "C" int tnvan_find_width_set(int n_spins, int n_edges, const int32_t* ei, const int32_t* ej, int w_u,
                                    int restarts, uint64_t seed, int mode, int anneal_iters, int32_t* out_w,
                                    int32_t* out_order, int32_t* out_info) {
  if (n_spins < 1 || n_spins > TNVAN_FIND_MAX_N || n_edges < 0 || (n_edges > 0 && (!ei || !ej)) || w_u < 0 ||
      restarts < 1 || mode < TNVAN_SLICE_FIXED || mode > TNVAN_SLICE_BEST || anneal_iters < 0 || !out_w ||
      !out_order || !out_info)
    return TNVAN_E_ARG;
  Graph G;
  G.n = n_spins;
  G.words = (n_spins + 63) / 64;
  G.bits.assign((size_t)G.n * G.words, 0);
  for (int k = 0; k < n_edges; ++k) {
    const int a = ei[k], b = ej[k];
    if (a < 0 || b < 0 || a >= n_spins || b >= n_spins || a == b) return TNVAN_E_ARG;
    G.set(a, b);
    G.set(b, a);
  }
  Result best;
  int best_tag = -1;
  for (int t = 0; t < restarts; ++t) {
    for (int m = TNVAN_SLICE_FIXED; m <= TNVAN_SLICE_GREEDY; ++m) {
      if (!(mode & m)) continue;
      Rng rng{seed ^ (0x632be59bd9b4e019ull * (uint64_t)(2 * t + m))};
      Result r = m == TNVAN_SLICE_FIXED ? search_fixed(G, w_u, rng) : search_greedy(G, w_u, rng);
      if (best_tag < 0 || r.W.size() < best.W.size()) {
        best = std::move(r);
        best_tag = 2 * t + (m == TNVAN_SLICE_GREEDY);
      }
    }
  }
  if (anneal_iters > 0) {
    Rng rng{seed ^ 0x5851f42d4c957f2dull};
    best = search_anneal(G, w_u, rng, best, anneal_iters, 0.5);
  }
  std::copy(best.W.begin(), best.W.end(), out_w);
  std::copy(best.order.begin(), best.order.end(), out_order);
  out_info[0] = (int32_t)best.W.size();
  out_info[1] = best.width;
  out_info[2] = best_tag;
  return TNVAN_OK;
}
