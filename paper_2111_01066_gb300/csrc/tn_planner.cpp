// Host planner: network simplification, contraction-order search, index
// slicing, slice batching and the device step program (paper, SI TN section and
// main text section II).  Host only: no CUDA call is made here.
#include <algorithm>
#include <bitset>
#include <cmath>
#include <array>
#include <cstring>
#include <functional>
#include <iterator>
#include <limits>
#include <memory>
#include <new>
#include <numeric>
#include <random>
#include <thread>
#include <unordered_map>

#include "tn_internal.h"

namespace tnx {
namespace {

constexpr int MAXW = 4096;
using WS = std::bitset<MAXW>;
// complex MACs charged per complex64 element moved (tn_plan_opts.mem_weight;
// set for the duration of one build_plan on its thread)
thread_local double g_alpha = 32.0;

double pow2(int e) { return std::ldexp(1.0, e); }

// ====================================================================== simplification
// SI, TN section: rank-1 and rank-2 tensors are absorbed into neighbours, and
// two tensors are pre-contracted when the result's rank is not larger than the
// larger input's.  Ranks count planning wires only: the closed output wires
// ("fixed") are set per batch by the leaf-select kernel and never enter a
// per-slice tensor.
struct Simplified {
  std::vector<HTensor> leaves;   // wires: planning wires first, then fixed wires
  std::vector<char> fixed;       // per network wire id
  std::vector<std::vector<int>> gates;   // per leaf: the circuit gates absorbed into it
};

Simplified simplify(const Network& net, uint64_t open_mask, const std::vector<int>& forced) {
  Simplified out;
  const int n = net.n_qubits;
  const int nw = (int)net.labels.size();
  std::vector<HTensor> ts = net.gates;
  std::vector<std::vector<int>> members(ts.size());   // circuit gates held by each tensor
  for (size_t g = 0; g < ts.size(); ++g) members[g] = {(int)g};
  // initial state |0> on every input wire
  for (int q = 0; q < n; ++q) {
    const int w = net.input_wire[q];
    if (net.gates_per_qubit[q] == 0) {
      HTensor t;   // a qubit with no gate: |0> sits directly on its output wire
      t.wires = {w};
      t.data = {cd(1, 0), cd(0, 0)};
      ts.push_back(std::move(t));
      members.emplace_back();
      continue;
    }
    for (auto& t : ts)
      if (std::find(t.wires.begin(), t.wires.end(), w) != t.wires.end()) {
        t = hfix(t, w, 0);
        break;
      }
  }
  out.fixed.assign(nw, 0);
  for (int q = 0; q < n; ++q)
    if (!((open_mask >> q) & 1)) out.fixed[net.output_wire[q]] = 1;
  // caller-sliced wires are fixed per slice: kept as leaf indices, never planned
  for (int w : forced) out.fixed[w] = 1;
  auto prank = [&](const HTensor& t) {
    int r = 0;
    for (int w : t.wires) r += !out.fixed[w];
    return r;
  };
  std::vector<char> alive(ts.size(), 1);
  auto owners = [&]() {
    std::vector<std::vector<int>> own(nw);
    for (size_t i = 0; i < ts.size(); ++i)
      if (alive[i])
        for (int w : ts[i].wires)
          if (!out.fixed[w]) own[w].push_back((int)i);
    return own;
  };
  auto n_alive = [&]() { return (int)std::count(alive.begin(), alive.end(), 1); };
  bool changed = true;
  while (changed && n_alive() > 1) {
    changed = false;
    auto own = owners();
    // (a) absorb rank <= 2 tensors into their highest-rank neighbour
    for (size_t i = 0; i < ts.size() && n_alive() > 1; ++i) {
      if (!alive[i] || prank(ts[i]) > 2) continue;
      int best = -1, best_rank = -1;
      for (int w : ts[i].wires) {
        if (out.fixed[w]) continue;
        for (int j : own[w])
          if (j != (int)i && alive[j] && prank(ts[j]) > best_rank) {
            best = j;
            best_rank = prank(ts[j]);
          }
      }
      if (best < 0) {
        // disconnected piece: fold it into the largest other tensor as an outer product
        for (size_t j = 0; j < ts.size(); ++j)
          if (j != i && alive[j] && prank(ts[j]) > best_rank) {
            best = (int)j;
            best_rank = prank(ts[j]);
          }
        if (best < 0) continue;
      }
      ts[best] = hcontract(ts[best], ts[i], &out.fixed);
      members[best].insert(members[best].end(), members[i].begin(), members[i].end());
      alive[i] = 0;
      changed = true;
      own = owners();
    }
    // (b) pre-contract pairs whose result is not larger than the larger input
    for (int w = 0; w < nw; ++w) {
      if (own[w].size() != 2) continue;
      const int a = own[w][0], b = own[w][1];
      if (!alive[a] || !alive[b] || a == b) continue;
      std::vector<int> uni;
      int shared = 0;
      for (int x : ts[a].wires)
        if (!out.fixed[x]) uni.push_back(x);
      for (int x : ts[b].wires) {
        if (out.fixed[x]) continue;
        if (std::find(uni.begin(), uni.end(), x) != uni.end())
          ++shared;
        else
          uni.push_back(x);
      }
      const int rc = (int)uni.size() - shared;
      if (rc <= std::max(prank(ts[a]), prank(ts[b]))) {
        ts[a] = hcontract(ts[a], ts[b], &out.fixed);
        members[a].insert(members[a].end(), members[b].begin(), members[b].end());
        alive[b] = 0;
        changed = true;
        own = owners();
      }
    }
  }
  for (size_t i = 0; i < ts.size(); ++i) {
    if (!alive[i]) continue;
    std::vector<int> order;
    for (int w : ts[i].wires)
      if (!out.fixed[w]) order.push_back(w);
    for (int w : ts[i].wires)
      if (out.fixed[w]) order.push_back(w);
    out.leaves.push_back(hpermute(ts[i], order));
    std::sort(members[i].begin(), members[i].end());
    out.gates.push_back(members[i]);
  }
  return out;
}

// ====================================================================== trees
struct Tree {
  int L = 0;
  std::vector<std::pair<int, int>> merges;  // merge i creates node L + i
  std::vector<WS> sets;                     // planning-wire set of each node
};

struct CostModel {
  // cost of one pairwise step from log2 sizes: MACs + ALPHA * elements moved
  static double step(int u, int a, int b, int c) {
    return pow2(u) + g_alpha * (pow2(a) + pow2(b) + pow2(c));
  }
};

double tree_cost(const Tree& t, const WS& sl) {
  double c = 0;
  WS keep = ~sl;
  for (size_t i = 0; i < t.merges.size(); ++i) {
    const WS& a = t.sets[t.merges[i].first];
    const WS& b = t.sets[t.merges[i].second];
    const WS& r = t.sets[t.L + i];
    c += CostModel::step((int)((a | b) & keep).count(), (int)(a & keep).count(),
                         (int)(b & keep).count(), (int)(r & keep).count());
  }
  return c;
}

// --------------------------------------------------------- exhaustive small subtrees
// Optimal order of <= 8 nodes by dynamic programming over subsets (the SI's
// brute-force optimisation of small subtrees).  Wires are mapped to a local
// 128-bit mask.
using u128 = unsigned __int128;
static inline int pc128(u128 x) {
  return __builtin_popcountll((uint64_t)x) + __builtin_popcountll((uint64_t)(x >> 64));
}

int dp_subtree(Tree& t, const std::vector<int>& nodes) {
  const int k = (int)nodes.size();
  if (k == 1) return nodes[0];
  // local wire index
  std::vector<int> wires;
  for (int v : nodes)
    for (size_t w = t.sets[v]._Find_first(); w < MAXW; w = t.sets[v]._Find_next(w))
      if (std::find(wires.begin(), wires.end(), (int)w) == wires.end()) wires.push_back((int)w);
  if (wires.size() > 128 || k > 10) {
    // fall back to a left-deep chain
    int cur = nodes[0];
    for (int i = 1; i < k; ++i) {
      t.merges.push_back({cur, nodes[i]});
      t.sets.push_back(t.sets[cur] ^ t.sets[nodes[i]]);
      cur = (int)t.sets.size() - 1;
    }
    return cur;
  }
  std::vector<u128> loc(k, 0);
  for (int i = 0; i < k; ++i)
    for (size_t j = 0; j < wires.size(); ++j)
      if (t.sets[nodes[i]].test(wires[j])) loc[i] |= (u128)1 << j;
  const int full = (1 << k) - 1;
  std::vector<u128> legs(full + 1, 0);
  for (int m = 1; m <= full; ++m) {
    const int lo = __builtin_ctz(m);
    legs[m] = legs[m & (m - 1)] ^ loc[lo];
  }
  std::vector<double> best(full + 1, std::numeric_limits<double>::infinity());
  std::vector<int> split(full + 1, 0);
  for (int i = 0; i < k; ++i) best[1 << i] = 0;
  for (int m = 1; m <= full; ++m) {
    if ((m & (m - 1)) == 0) continue;
    const int lo = m & -m;
    // enumerate submasks containing the lowest bit to avoid double counting
    for (int s = (m - 1) & m; s > 0; s = (s - 1) & m) {
      if (!(s & lo)) continue;
      const int r = m ^ s;
      const double c = best[s] + best[r] +
                       CostModel::step(pc128(legs[s] | legs[r]), pc128(legs[s]), pc128(legs[r]),
                                       pc128(legs[m]));
      if (c < best[m]) {
        best[m] = c;
        split[m] = s;
      }
    }
  }
  std::function<int(int)> emit = [&](int m) -> int {
    if ((m & (m - 1)) == 0) return nodes[__builtin_ctz(m)];
    const int a = emit(split[m]);
    const int b = emit(m ^ split[m]);
    t.merges.push_back({a, b});
    t.sets.push_back(t.sets[a] ^ t.sets[b]);
    return (int)t.sets.size() - 1;
  };
  return emit(full);
}

// --------------------------------------------------------- recursive bisection
// The SI partitions the network into subtrees with a hypergraph partitioner
// before slicing and re-optimising small subtrees.  Here: balanced bisection by
// region growing plus Fiduccia-Mattheyses refinement, minimising the number of
// wires cut, recursively, with exhaustive search below a leaf-cluster size.
struct Bisector {
  const std::vector<std::vector<std::pair<int, int>>>& adj;  // leaf -> (nbr, multiplicity)
  std::mt19937_64& rng;
  double eps;
  int leafmax;
  int inits;

  std::vector<char> partition(const std::vector<int>& nodes) {
    const int n = (int)nodes.size();
    std::unordered_map<int, int> loc;
    for (int i = 0; i < n; ++i) loc[nodes[i]] = i;
    std::vector<std::vector<std::pair<int, int>>> ladj(n);
    for (int i = 0; i < n; ++i)
      for (auto [v, m] : adj[nodes[i]]) {
        auto it = loc.find(v);
        if (it != loc.end()) ladj[i].push_back({it->second, m});
      }
    std::uniform_real_distribution<double> U(0.0, 1.0);
    std::vector<char> best_side;
    int best_cut = std::numeric_limits<int>::max();
    const int lo = std::max(1, (int)std::floor(n * (0.5 - eps)));
    const int hi = std::min(n - 1, (int)std::ceil(n * (0.5 + eps)));
    for (int trial = 0; trial < inits; ++trial) {
      std::vector<char> side(n, 1);
      const int target = std::min(hi, lo + (int)(U(rng) * (hi - lo + 1)));
      // region growing from a random seed
      int count = 0;
      std::vector<int> queue;
      std::vector<char> seen(n, 0);
      while (count < target) {
        if (queue.empty()) {
          std::vector<int> cand;
          for (int i = 0; i < n; ++i)
            if (!seen[i]) cand.push_back(i);
          if (cand.empty()) break;
          const int s = cand[(size_t)(U(rng) * cand.size()) % cand.size()];
          seen[s] = 1;
          queue.push_back(s);
        }
        const int v = queue.front();
        queue.erase(queue.begin());
        side[v] = 0;
        ++count;
        for (auto [u, m] : ladj[v])
          if (!seen[u]) {
            seen[u] = 1;
            queue.push_back(u);
          }
      }
      // FM passes
      auto cut_of = [&]() {
        int c = 0;
        for (int i = 0; i < n; ++i)
          for (auto [u, m] : ladj[i])
            if (side[i] != side[u]) c += m;
        return c / 2;
      };
      int cur = cut_of();
      for (int pass = 0; pass < 8; ++pass) {
        std::vector<int> gain(n, 0);
        for (int i = 0; i < n; ++i)
          for (auto [u, m] : ladj[i]) gain[i] += (side[i] != side[u]) ? m : -m;
        std::vector<char> locked(n, 0);
        int cnt0 = 0;
        for (int i = 0; i < n; ++i) cnt0 += side[i] == 0;
        std::vector<int> moved;
        std::vector<int> cuts;
        int c = cur;
        for (int step = 0; step < n; ++step) {
          int bv = -1;
          double bg = -1e18;
          for (int i = 0; i < n; ++i) {
            if (locked[i]) continue;
            const int c0 = cnt0 + (side[i] == 0 ? -1 : 1);
            if (c0 < lo || c0 > hi) continue;
            const double g = gain[i] + 1e-3 * U(rng);
            if (g > bg) {
              bg = g;
              bv = i;
            }
          }
          if (bv < 0) break;
          c -= gain[bv];
          cnt0 += side[bv] == 0 ? -1 : 1;
          side[bv] ^= 1;
          locked[bv] = 1;
          gain[bv] = -gain[bv];
          for (auto [u, m] : ladj[bv]) gain[u] += (side[u] != side[bv]) ? 2 * m : -2 * m;
          moved.push_back(bv);
          cuts.push_back(c);
        }
        int bi = -1, bc = cur;
        for (size_t s = 0; s < cuts.size(); ++s)
          if (cuts[s] < bc) {
            bc = cuts[s];
            bi = (int)s;
          }
        for (int s = (int)moved.size() - 1; s > bi; --s) side[moved[s]] ^= 1;
        if (bi < 0) break;
        cur = bc;
      }
      if (cur < best_cut) {
        best_cut = cur;
        best_side = side;
      }
    }
    return best_side;
  }

  int build(Tree& t, const std::vector<int>& nodes) {
    if ((int)nodes.size() <= leafmax) return dp_subtree(t, nodes);
    auto side = partition(nodes);
    std::vector<int> p0, p1;
    for (size_t i = 0; i < nodes.size(); ++i) (side[i] ? p1 : p0).push_back(nodes[i]);
    if (p0.empty() || p1.empty()) {
      p0.assign(nodes.begin(), nodes.begin() + nodes.size() / 2);
      p1.assign(nodes.begin() + nodes.size() / 2, nodes.end());
    }
    const int a = build(t, p0);
    const int b = build(t, p1);
    t.merges.push_back({a, b});
    t.sets.push_back(t.sets[a] ^ t.sets[b]);
    return (int)t.sets.size() - 1;
  }
};

// --------------------------------------------------------- subtree reconfiguration
// Re-optimise every subtree of up to 8 frontier nodes exhaustively (SI: small
// subtrees are optimised by brute force) with the sliced wires removed.
void reconfigure(Tree& t, const WS& sl, int passes) {
  for (int pass = 0; pass < passes; ++pass) {
    bool improved = false;
    const int nm = (int)t.merges.size();
    for (int root = t.L + nm - 1; root >= t.L; --root) {
      // collect the frontier by expanding the costliest internal node
      std::vector<int> frontier = {root};
      std::vector<int> internal;
      while ((int)frontier.size() < 8) {
        int best = -1;
        double bc = -1;
        for (size_t i = 0; i < frontier.size(); ++i) {
          const int v = frontier[i];
          if (v < t.L) continue;
          const auto [a, b] = t.merges[v - t.L];
          const double c = pow2((int)((t.sets[a] | t.sets[b]) & ~sl).count());
          if (c > bc) {
            bc = c;
            best = (int)i;
          }
        }
        if (best < 0) break;
        const int v = frontier[best];
        frontier.erase(frontier.begin() + best);
        internal.push_back(v);
        frontier.push_back(t.merges[v - t.L].first);
        frontier.push_back(t.merges[v - t.L].second);
      }
      if (frontier.size() < 3) continue;
      double old_cost = 0;
      for (int v : internal) {
        const auto [a, b] = t.merges[v - t.L];
        old_cost += CostModel::step((int)((t.sets[a] | t.sets[b]) & ~sl).count(),
                                    (int)(t.sets[a] & ~sl).count(), (int)(t.sets[b] & ~sl).count(),
                                    (int)(t.sets[v] & ~sl).count());
      }
      // exhaustive re-optimisation in a scratch tree that shares the node sets
      Tree s;
      s.L = 0;
      s.sets = t.sets;
      for (auto& w : s.sets) w &= ~sl;
      const size_t base = s.sets.size();
      dp_subtree(s, frontier);
      double new_cost = 0;
      for (size_t i = 0; i < s.merges.size(); ++i) {
        const auto [a, b] = s.merges[i];
        new_cost += CostModel::step((int)(s.sets[a] | s.sets[b]).count(), (int)s.sets[a].count(),
                                    (int)s.sets[b].count(), (int)s.sets[base + i].count());
      }
      if (new_cost < old_cost * 0.999 && s.merges.size() == internal.size()) {
        // rewrite: reuse the internal node ids, the subtree root keeps its id
        std::vector<int> others;
        for (int v : internal)
          if (v != root) others.push_back(v);
        std::sort(others.begin(), others.end());
        std::unordered_map<int, int> remap;  // scratch id -> tree id
        for (size_t i = 0; i < s.merges.size(); ++i) {
          int a = s.merges[i].first, b = s.merges[i].second;
          if (a >= (int)base) a = remap[a];
          if (b >= (int)base) b = remap[b];
          const int id = (i + 1 == s.merges.size()) ? root : others[i];
          remap[(int)(base + i)] = id;
          t.merges[id - t.L] = {a, b};
          t.sets[id] = t.sets[a] ^ t.sets[b];
        }
        improved = true;
      }
    }
    if (!improved) break;
  }
}

// Topological order of merges (children before parents), deepest-first so that
// the larger subtree runs before its sibling.
std::vector<int> post_order(const Tree& t) {
  std::vector<int> order;
  const int root = t.L + (int)t.merges.size() - 1;
  std::vector<std::pair<int, int>> stack = {{root, 0}};
  while (!stack.empty()) {
    auto& [v, state] = stack.back();
    if (v < t.L) {
      stack.pop_back();
      continue;
    }
    if (state == 0) {
      state = 1;
      const auto [a, b] = t.merges[v - t.L];
      stack.push_back({b, 0});
      stack.push_back({a, 0});
    } else {
      order.push_back(v - t.L);
      stack.pop_back();
    }
  }
  return order;
}

// Work for all 2^S slices when every node is computed once per distinct value
// of the sliced wires it depends on (the executor shares slice-independent
// parts of a chunk's slices and runs slice-free subtrees once):
// sum over steps of 2^|sliced wires below it| x its per-slice cost.
double reuse_cost(const Tree& t, const WS& sl) {
  if (t.merges.empty()) return 0.0;
  const WS keep = ~sl;
  std::vector<WS> dep(t.sets.size());
  for (int i = 0; i < t.L; ++i) dep[i] = t.sets[i] & sl;
  double c = 0;
  for (int i : post_order(t)) {
    const int x = t.merges[i].first, y = t.merges[i].second;
    dep[t.L + i] = dep[x] | dep[y];
    const WS& a = t.sets[x];
    const WS& b = t.sets[y];
    const WS& r = t.sets[t.L + i];
    c += std::ldexp(CostModel::step((int)((a | b) & keep).count(), (int)(a & keep).count(),
                                    (int)(b & keep).count(), (int)(r & keep).count()),
                    (int)dep[t.L + i].count());
  }
  return c;
}

// --------------------------------------------------------- slicing
// Main text, section II: slice wires until every intermediate fits the bound;
// each pick minimises the total cost 2^S * cost(per slice).
std::vector<int> choose_slices(const Tree& t, const WS& open, int bound, int min_slices) {
  std::vector<int> out;
  WS sl;
  const int nm = (int)t.merges.size();
  while (true) {
    int mx = 0;
    for (const auto& s : t.sets) mx = std::max(mx, (int)(s & ~sl).count());
    if (mx <= bound && (int)out.size() >= min_slices) break;
    WS cand;
    const int thresh = mx > bound ? mx : std::max(0, mx - 3);
    for (const auto& s : t.sets)
      if ((int)(s & ~sl).count() >= thresh) cand |= s;
    cand &= ~sl;
    cand &= ~open;
    if (cand.none()) fail(TN_ERR_PLAN, "no wire left to slice (open qubits exceed the bound?)");
    std::vector<int> ua(nm), ub(nm), uc(nm), uu(nm);
    for (int i = 0; i < nm; ++i) {
      const WS& a = t.sets[t.merges[i].first];
      const WS& b = t.sets[t.merges[i].second];
      ua[i] = (int)(a & ~sl).count();
      ub[i] = (int)(b & ~sl).count();
      uc[i] = (int)(t.sets[t.L + i] & ~sl).count();
      uu[i] = (int)((a | b) & ~sl).count();
    }
    int best_w = -1;
    double best_c = std::numeric_limits<double>::infinity();
    int best_mx = 1 << 30;
    for (size_t w = cand._Find_first(); w < MAXW; w = cand._Find_next(w)) {
      double c = 0;
      for (int i = 0; i < nm; ++i) {
        const WS& a = t.sets[t.merges[i].first];
        const WS& b = t.sets[t.merges[i].second];
        const bool ia = a.test(w), ib = b.test(w);
        c += CostModel::step(uu[i] - (ia || ib), ua[i] - ia, ub[i] - ib, uc[i] - t.sets[t.L + i].test(w));
      }
      // prefer picks that lower the maximum when over the bound
      int nmx = 0;
      if (mx > bound)
        for (const auto& s : t.sets) nmx = std::max(nmx, (int)(s & ~sl).count() - (int)s.test(w));
      if (nmx < best_mx || (nmx == best_mx && c < best_c)) {
        best_mx = nmx;
        best_c = c;
        best_w = (int)w;
      }
    }
    sl.set(best_w);
    out.push_back(best_w);
    if (out.size() > 60) fail(TN_ERR_PLAN, "slicing did not converge under 60 wires");
  }
  return out;
}

}  // namespace

// ====================================================================== plan builder
Plan* build_plan(const Network& net, const tn_plan_opts& o) {
  if (o.max_log2_intermediate < 1 || o.max_log2_intermediate > 36)
    fail(TN_ERR_ARG, "max_log2_intermediate must be in [1, 36]");
  if (o.precision < TN_PREC_FP32 || o.precision > TN_PREC_FP16X3) fail(TN_ERR_ARG, "unknown precision");
  if (o.complex_mult != 3 && o.complex_mult != 4) fail(TN_ERR_ARG, "complex_mult must be 3 or 4");
  if (o.complex_mult == 3 && o.precision == TN_PREC_FP32)
    fail(TN_ERR_UNSUPPORTED, "the FP32 CUDA-core path forms 4M products only; 3M needs TF32 or BF16X3");
  if (o.min_log2_slices < 0 || o.min_log2_slices > 48) fail(TN_ERR_ARG, "min_log2_slices out of range");
  const int n = net.n_qubits;
  if (n < 64 && (o.open_mask >> n) != 0) fail(TN_ERR_ARG, "open_mask names a qubit >= n_qubits");
  auto* P = new Plan;
  std::unique_ptr<Plan> guard(P);
  P->opts = o;
  P->n_qubits = n;
  for (int q = 0; q < n; ++q)
    if ((o.open_mask >> q) & 1) P->open_qubits.push_back(q);
  const int k_open = (int)P->open_qubits.size();
  if (k_open > o.max_log2_intermediate) fail(TN_ERR_PLAN, "open qubits alone exceed the bound");
  if (k_open > 30) fail(TN_ERR_UNSUPPORTED, "more than 30 open qubits");

  // caller-chosen slices: internal wires (q, t), 1 <= t < gates on q
  std::vector<int> forced;
  std::vector<int> forced_bit(net.labels.size(), -1);
  if (o.n_forced_slices < 0 || o.n_forced_slices > 48) fail(TN_ERR_ARG, "n_forced_slices out of range");
  if (o.n_forced_slices > 0 && (!o.forced_slice_qubit || !o.forced_slice_t))
    fail(TN_ERR_ARG, "forced slice arrays are NULL");
  for (int j = 0; j < o.n_forced_slices; ++j) {
    const int q = o.forced_slice_qubit[j], t = o.forced_slice_t[j];
    if (q < 0 || q >= n || t < 1 || t >= net.gates_per_qubit[q])
      fail(TN_ERR_ARG, "forced slice (" + std::to_string(q) + ", " + std::to_string(t) + ") is not an internal wire");
    int w = -1;
    for (size_t i = 0; i < net.labels.size(); ++i)
      if (net.labels[i].q == q && net.labels[i].t == t) w = (int)i;
    if (w < 0 || forced_bit[w] >= 0) fail(TN_ERR_ARG, "forced slice wire missing or repeated");
    forced_bit[w] = j;
    forced.push_back(w);
    P->sliced.push_back(net.labels[w]);
  }
  const int nF = (int)forced.size();
  Simplified S = simplify(net, o.open_mask, forced);
  const int L = (int)S.leaves.size();
  P->n_leaves = L;
  P->leaf_gates = S.gates;

  // planning wire numbering
  std::vector<int> pw_of(net.labels.size(), -1);
  std::vector<int> wire_of_pw;
  for (const auto& lf : S.leaves)
    for (int w : lf.wires)
      if (!S.fixed[w] && pw_of[w] < 0) {
        pw_of[w] = (int)wire_of_pw.size();
        wire_of_pw.push_back(w);
      }
  const int W = (int)wire_of_pw.size();
  if (W > MAXW) fail(TN_ERR_UNSUPPORTED, "network has more than 4096 wires after simplification");
  WS open_ws;
  for (int q : P->open_qubits)
    if (pw_of[net.output_wire[q]] >= 0) open_ws.set(pw_of[net.output_wire[q]]);

  Tree base;
  base.L = L;
  base.sets.resize(L);
  for (int i = 0; i < L; ++i)
    for (int w : S.leaves[i].wires)
      if (!S.fixed[w]) base.sets[i].set(pw_of[w]);
  // leaf adjacency
  std::vector<std::vector<std::pair<int, int>>> adj(L);
  {
    std::vector<std::vector<int>> own(W);
    for (int i = 0; i < L; ++i)
      for (size_t w = base.sets[i]._Find_first(); w < MAXW; w = base.sets[i]._Find_next(w))
        own[w].push_back(i);
    std::vector<std::unordered_map<int, int>> m(L);
    for (int w = 0; w < W; ++w)
      if (own[w].size() == 2) {
        m[own[w][0]][own[w][1]]++;
        m[own[w][1]][own[w][0]]++;
      }
    for (int i = 0; i < L; ++i)
      for (auto& [j, c] : m[i]) adj[i].push_back({j, c});
    for (auto& v : adj) std::sort(v.begin(), v.end());
  }

  // order search: randomised recursive bisection trials, each sliced to the bound
  const int trials = o.trials > 0 ? o.trials : 64;
  const int bound = o.max_log2_intermediate;
  Tree best_tree;
  std::vector<int> best_sl;
  double best_total = std::numeric_limits<double>::infinity();
  std::vector<int> all(L);
  std::iota(all.begin(), all.end(), 0);
  // Trials are independent (trial tr draws from seed * 1000003 + tr) and run
  // on all host cores; the best by reuse-aware work wins, ties to the lowest
  // trial index, so the result does not depend on the thread count.
  struct TrialResult {
    double total = std::numeric_limits<double>::infinity();
    Tree tree;
    std::vector<int> sl;
  };
  std::vector<TrialResult> res(trials);
  auto run_trial = [&](int tr) {
    std::mt19937_64 rng(o.seed * 1000003ULL + (uint64_t)tr);
    const double eps_choices[4] = {0.05, 0.12, 0.2, 0.3};
    Bisector bis{adj, rng, eps_choices[(tr / 2) % 4], (tr % 2) ? 6 : 8, 3};
    Tree t = base;
    if (L > 1) bis.build(t, all);
    std::vector<int> sl = (L > 1) ? choose_slices(t, open_ws, bound, o.min_log2_slices) : std::vector<int>{};
    WS slw;
    for (int w : sl) slw.set(w);
    res[tr].total = reuse_cost(t, slw);
    res[tr].tree = std::move(t);
    res[tr].sl = std::move(sl);
  };
  {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nth = (int)std::min<unsigned>(hw, (unsigned)trials);
    const double alpha = g_alpha;
    std::vector<std::exception_ptr> errs(nth);
    std::vector<std::thread> pool;
    for (int th = 0; th < nth; ++th)
      pool.emplace_back([&, th]() {
        g_alpha = alpha;
        try {
          for (int tr = th; tr < trials; tr += nth) run_trial(tr);
        } catch (...) {
          errs[th] = std::current_exception();
        }
      });
    for (auto& t : pool) t.join();
    for (auto& e : errs)
      if (e) std::rethrow_exception(e);
  }
  // subtree reconfiguration with the slices in place (then re-slicing) on the
  // best few trials, in parallel: its gains vary a lot from tree to tree, so
  // the best trial before it is not always the best after it
  if (L == 1 && o.min_log2_slices > 0) fail(TN_ERR_PLAN, "a single-tensor network cannot be sliced");
  std::vector<int> rank_tr(trials);
  std::iota(rank_tr.begin(), rank_tr.end(), 0);
  std::stable_sort(rank_tr.begin(), rank_tr.end(), [&](int x, int y) { return res[x].total < res[y].total; });
  const int n_reconf = L > 2 ? std::min(trials, 8) : 0;
  std::vector<TrialResult> rec(n_reconf);
  {
    const double alpha = g_alpha;
    std::vector<std::exception_ptr> errs(n_reconf);
    std::vector<std::thread> pool;
    for (int j = 0; j < n_reconf; ++j)
      pool.emplace_back([&, j]() {
        g_alpha = alpha;
        try {
          const TrialResult& r = res[rank_tr[j]];
          WS slw;
          for (int w : r.sl) slw.set(w);
          Tree t2 = r.tree;
          reconfigure(t2, slw, 3);
          std::vector<int> sl2 = choose_slices(t2, open_ws, bound, o.min_log2_slices);
          WS s2;
          for (int w : sl2) s2.set(w);
          rec[j].total = reuse_cost(t2, s2);
          rec[j].tree = std::move(t2);
          rec[j].sl = std::move(sl2);
        } catch (...) {
          errs[j] = std::current_exception();
        }
      });
    for (auto& t : pool) t.join();
    for (auto& e : errs)
      if (e) std::rethrow_exception(e);
  }
  // best of the trials and of their reconfigurations (ties: trials first, lower rank first)
  for (int tr = 0; tr < trials; ++tr)
    if (res[tr].total < best_total) {
      best_total = res[tr].total;
      best_tree = res[tr].tree;
      best_sl = res[tr].sl;
    }
  for (int j = 0; j < n_reconf; ++j)
    if (rec[j].total < best_total) {
      best_total = rec[j].total;
      best_tree = rec[j].tree;
      best_sl = rec[j].sl;
    }
  Tree& T = best_tree;
  WS SL;
  for (int w : best_sl) SL.set(w);
  const int nS = (int)best_sl.size();
  const int nm = (int)T.merges.size();

  const std::vector<int> order = (nm > 0) ? post_order(T) : std::vector<int>{};
  // dependence of every node on the sliced wires (through its subtree's leaves)
  std::vector<WS> dep(T.sets.size());
  for (int i = 0; i < L; ++i) dep[i] = T.sets[i] & SL;
  for (int i : order) dep[L + i] = dep[T.merges[i].first] | dep[T.merges[i].second];

  // batch bits: choose which sliced wires vary inside a chunk
  auto chunk_cost = [&](const WS& B) {
    double c = 0;
    for (int i = 0; i < nm; ++i) {
      const WS& a = T.sets[T.merges[i].first];
      const WS& b = T.sets[T.merges[i].second];
      const int mult = (int)(dep[L + i] & B).count();
      c += pow2(mult) * CostModel::step((int)((a | b) & ~SL).count(), (int)(a & ~SL).count(),
                                        (int)(b & ~SL).count(), (int)(T.sets[L + i] & ~SL).count());
    }
    return c;
  };
  std::vector<int> order_sl;  // slice bit order: batch bits first
  {
    WS B;
    std::vector<int> rest = best_sl;
    const int bmax = std::min(nS, 12);
    for (int j = 0; j < bmax; ++j) {
      int bw = -1;
      double bc = std::numeric_limits<double>::infinity();
      for (int w : rest) {
        WS B2 = B;
        B2.set(w);
        const double c = chunk_cost(B2);
        if (c < bc) {
          bc = c;
          bw = w;
        }
      }
      B.set(bw);
      order_sl.push_back(bw);
      rest.erase(std::find(rest.begin(), rest.end(), bw));
    }
    for (int w : rest) order_sl.push_back(w);
  }
  std::vector<int> slice_bit(W, -1);
  for (int j = 0; j < nS; ++j) slice_bit[order_sl[j]] = nF + j;
  for (int j = 0; j < nS; ++j) P->sliced.push_back(net.labels[wire_of_pw[order_sl[j]]]);

  // ------------------------------------------------ step program for a given b
  struct NodeInfo {
    std::vector<int> wires;  // planning wires (unsliced), storage order
    uint32_t bmask = 0;
    std::vector<int> border;  // batch bits (chunk slice bits) in storage order, above the wires
    int64_t off = -1;
  };
  auto elems_of = [](const NodeInfo& ni) {
    return (int64_t)1 << (ni.wires.size() + __builtin_popcount(ni.bmask));
  };
  const int64_t cap_bytes = o.max_arena_bytes > 0 ? o.max_arena_bytes : (int64_t)96 << 30;
  std::vector<std::vector<int>> node_order;   // storage order of every node's wires
  std::vector<std::vector<int>> border_of;    // and of its batch bits
  // Dependence of every tree node on the slice id (bit 0) and on the closed
  // output bits (bit 1).  Results of steps with flags 0 (the same in every
  // chunk of every call) or 2 (the same in every chunk of one batch) are
  // computed once, by a prologue; those that a later-class step (or the root
  // sum) reads stay in a persistent pool at the start of the arena.
  std::vector<int> nflag(L + nm, 0), parent(L + nm, -1);
  for (int i = 0; i < L; ++i)
    for (int w : S.leaves[i].wires) {
      if (!S.fixed[w] && SL.test(pw_of[w])) nflag[i] |= 1;
      if (S.fixed[w]) nflag[i] |= forced_bit[w] >= 0 ? 1 : 2;
    }
  for (int mi : order) {
    nflag[L + mi] = nflag[T.merges[mi].first] | nflag[T.merges[mi].second];
    parent[T.merges[mi].first] = L + mi;
    parent[T.merges[mi].second] = L + mi;
  }
  std::vector<char> pooled(L + nm, 0);
  for (int mi : order) {
    const int v = L + mi;
    if ((nflag[v] & 1) == 0 && (parent[v] < 0 || nflag[parent[v]] != nflag[v])) pooled[v] = 1;
  }
  std::vector<int> exec_group;   // group id of every step in execution order (-1: none)
  auto layout = [&](int b, std::vector<NodeInfo>& info, std::vector<StepDesc>& steps,
                    int64_t& arena, std::vector<int>& exec) -> bool {
    info.assign(L + nm, NodeInfo{});
    for (int i = 0; i < L; ++i) {
      for (int w : S.leaves[i].wires)
        if (!S.fixed[w] && !SL.test(pw_of[w])) info[i].wires.push_back(pw_of[w]);
      for (int w : S.leaves[i].wires)
        if (!S.fixed[w] && SL.test(pw_of[w]) && slice_bit[pw_of[w]] < b)
          info[i].bmask |= 1u << slice_bit[pw_of[w]];
    }
    // Layout pass (SI figure S7a: C is written in the index order its consumer
    // wants), from the root down.  The streamed operand A of every step is stored
    // as [contracted wires..., free wires..., free batch bits..., shared batch
    // bits...]: a row-major matrix whose rows (the free wires, then the batch
    // bits folded into them) are contiguous, so the GEMM fetches its tiles with
    // the tensor memory accelerator.  Inside that frame the order is free and is
    // chosen for the two kernels that touch the tensor: the free part follows the
    // order of those wires in the step's result (tile rows then run along C's
    // memory order), and the contracted part lists first the rows of the step
    // that produces A (its 32-row warps then write contiguous runs).  A tensor
    // that is no step's A keeps its producer's order: rows, then columns.
    {
      std::vector<std::vector<int>> wset(L + nm);
      std::vector<uint32_t> bm(L + nm, 0);
      std::vector<int> a_of(nm, -1), b_of(nm, -1);
      for (int i = 0; i < L; ++i) {
        wset[i] = info[i].wires;
        std::sort(wset[i].begin(), wset[i].end());
        bm[i] = info[i].bmask;
      }
      for (int mi : order) {
        const int x = T.merges[mi].first, y = T.merges[mi].second;
        std::vector<int> u;
        std::set_symmetric_difference(wset[x].begin(), wset[x].end(), wset[y].begin(), wset[y].end(),
                                      std::back_inserter(u));
        wset[L + mi] = u;
        bm[L + mi] = bm[x] | bm[y];
        const int64_t ex = (int64_t)1 << (wset[x].size() + __builtin_popcount(bm[x]));
        const int64_t ey = (int64_t)1 << (wset[y].size() + __builtin_popcount(bm[y]));
        const bool x_is_a = ex > ey || (ex == ey && wset[x].size() >= wset[y].size());
        a_of[mi] = x_is_a ? x : y;
        b_of[mi] = x_is_a ? y : x;
      }
      auto has = [&](int node, int w) { return std::binary_search(wset[node].begin(), wset[node].end(), w); };
      std::vector<std::vector<int>> lw(L + nm), lb(L + nm);
      std::vector<char> lset(L + nm, 0);
      for (auto it = order.rbegin(); it != order.rend(); ++it) {
        const int mi = *it, c = L + mi, a = a_of[mi], bb = b_of[mi];
        std::vector<int> k, m, n;
        for (int w : wset[a]) (has(bb, w) ? k : m).push_back(w);
        for (int w : wset[bb])
          if (!has(a, w)) n.push_back(w);
        std::vector<int> fb, sb, nbits;  // A-only, shared and B-only batch bits
        for (int j = 0; j < 32; ++j) {
          const bool ia = (bm[a] >> j) & 1, ib = (bm[bb] >> j) & 1;
          if (ia && ib) sb.push_back(j);
          else if (ia) fb.push_back(j);
          else if (ib) nbits.push_back(j);
        }
        if (lset[c]) {
          auto rank_in = [](const std::vector<int>& v, int x) {
            return (int)(std::find(v.begin(), v.end(), x) - v.begin());
          };
          std::stable_sort(m.begin(), m.end(),
                           [&](int u, int v) { return rank_in(lw[c], u) < rank_in(lw[c], v); });
          std::stable_sort(fb.begin(), fb.end(),
                           [&](int u, int v) { return rank_in(lb[c], u) < rank_in(lb[c], v); });
        }
        if (a >= L) {  // rows of A's producer first among the contracted wires
          const int pa = a_of[a - L], pb = b_of[a - L];
          std::stable_partition(k.begin(), k.end(), [&](int w) { return has(pa, w) && !has(pb, w); });
        }
        lw[a] = k;
        lw[a].insert(lw[a].end(), m.begin(), m.end());
        lb[a] = fb;
        lb[a].insert(lb[a].end(), sb.begin(), sb.end());
        lset[a] = 1;
        if (!lset[c]) {
          lw[c] = m;
          lw[c].insert(lw[c].end(), n.begin(), n.end());
          lb[c] = fb;
          lb[c].insert(lb[c].end(), nbits.begin(), nbits.end());
          lb[c].insert(lb[c].end(), sb.begin(), sb.end());
          lset[c] = 1;
        }
      }
      for (int i = 0; i < L; ++i) {
        if (lset[i]) {
          info[i].wires = lw[i];
          info[i].border = lb[i];
        } else {
          info[i].border.clear();
          for (int j = 0; j < 32; ++j)
            if ((info[i].bmask >> j) & 1) info[i].border.push_back(j);
        }
      }
      node_order.swap(lw);
      border_of.swap(lb);
      // Execution order.  First the steps that depend on neither the slice id
      // nor the closed output bits (run once per plan), in post-order; then
      // those that depend on the closed bits only (run once per batch); then
      // the slice-dependent ones (run in every chunk).  Within the last two
      // classes, the small steps (under 2^20 multiply-adds per chunk: the
      // CUDA-core kernels) whose subtree holds only such steps, leaves and
      // results of earlier classes come first, one group per dependency level
      // (a group's steps are independent and run as one launch); then the
      // other steps of the class in post-order, where the remaining small
      // steps are deferred and emitted the same way, level by level, right
      // before the first step that reads one of them.
      exec.clear();
      exec_group.clear();
      std::vector<char> pend(nm, 0), hoist(nm, 0);
      std::vector<int> pending, lev(nm, 0);
      int next_group = 0;
      auto small = [&](int mi) {
        const int x = T.merges[mi].first, y = T.merges[mi].second;
        std::vector<int> u;
        std::set_union(wset[x].begin(), wset[x].end(), wset[y].begin(), wset[y].end(), std::back_inserter(u));
        return (int)u.size() + __builtin_popcount(bm[x] | bm[y]) < 20;
      };
      // emit `set` (merge indices in post-order, closed under "child in set
      // comes first") as one group per level among them
      auto emit_levels = [&](const std::vector<int>& set, const std::vector<char>& in) {
        int maxl = 0;
        for (int mi : set) {
          int l = 0;
          for (int ch : {T.merges[mi].first, T.merges[mi].second})
            if (ch >= L && in[ch - L]) l = std::max(l, lev[ch - L]);
          lev[mi] = l + 1;
          maxl = std::max(maxl, l + 1);
        }
        for (int l = 1; l <= maxl; ++l) {
          for (int mi : set)
            if (lev[mi] == l) {
              exec.push_back(mi);
              exec_group.push_back(next_group);
            }
          ++next_group;
        }
      };
      for (int mi : order)
        if (nflag[L + mi] == 0) {
          exec.push_back(mi);
          exec_group.push_back(-1);
        }
      for (int cls : {2, 1}) {   // per batch, then per chunk (flags 1 or 3)
        auto in_cls = [&](int v) { return cls == 2 ? nflag[v] == 2 : (nflag[v] & 1) != 0; };
        std::vector<int> hoisted;
        for (int mi : order) {
          if (!in_cls(L + mi) || !small(mi)) continue;
          bool ok = true;
          for (int ch : {T.merges[mi].first, T.merges[mi].second})
            if (ch >= L && in_cls(ch) && !hoist[ch - L]) ok = false;
          if (ok) {
            hoist[mi] = 1;
            hoisted.push_back(mi);
          }
        }
        emit_levels(hoisted, hoist);
        auto flush = [&]() {
          emit_levels(pending, pend);
          for (int mi : pending) pend[mi] = 0;
          pending.clear();
        };
        for (int mi : order) {
          if (!in_cls(L + mi) || hoist[mi]) continue;
          if (small(mi)) {
            pending.push_back(mi);
            pend[mi] = 1;
            continue;
          }
          const int x = T.merges[mi].first, y = T.merges[mi].second;
          if ((x >= L && pend[x - L]) || (y >= L && pend[y - L])) flush();
          exec.push_back(mi);
          exec_group.push_back(-1);
        }
        flush();
      }
    }
    // best-fit arena allocator
    std::vector<std::pair<int64_t, int64_t>> freel;  // (offset, size)
    int64_t end = 0;
    const int64_t AL = 64;
    auto alloc = [&](int64_t sz) {
      sz = (sz + AL - 1) / AL * AL;
      int bi = -1;
      for (size_t i = 0; i < freel.size(); ++i)
        if (freel[i].second >= sz && (bi < 0 || freel[i].second < freel[bi].second)) bi = (int)i;
      if (bi >= 0) {
        const int64_t off = freel[bi].first;
        freel[bi].first += sz;
        freel[bi].second -= sz;
        if (freel[bi].second == 0) freel.erase(freel.begin() + bi);
        return off;
      }
      const int64_t off = end;
      end += sz;
      return off;
    };
    auto release = [&](int64_t off, int64_t sz) {
      sz = (sz + AL - 1) / AL * AL;
      freel.push_back({off, sz});
      std::sort(freel.begin(), freel.end());
      std::vector<std::pair<int64_t, int64_t>> merged;
      for (auto& f : freel) {
        if (!merged.empty() && merged.back().first + merged.back().second == f.first)
          merged.back().second += f.second;
        else
          merged.push_back(f);
      }
      freel.swap(merged);
      if (!freel.empty() && freel.back().first + freel.back().second == end) {
        end = freel.back().first;
        freel.pop_back();
      }
    };
    // the persistent pool first: one slot per pooled result (no batch bits: it
    // depends on no slice)
    std::vector<int64_t> pool_off(L + nm, -1);
    for (int mi : order)
      if (pooled[L + mi]) {
        pool_off[L + mi] = end;
        end += (((int64_t)1 << node_order[L + mi].size()) + AL - 1) / AL * AL;
      }
    int64_t peak = end;
    for (int i = 0; i < L; ++i) {
      info[i].off = alloc(elems_of(info[i]));
      peak = std::max(peak, end);
    }
    steps.clear();
    std::vector<int> step_of(nm, -1);
    // a group's outputs are all allocated before any of its operands is
    // released, so that no output overlaps an operand of another step of the group
    std::vector<std::pair<int64_t, int64_t>> to_release;
    for (size_t e = 0; e < exec.size(); ++e) {
      const int mi = exec[e];
      const int x = T.merges[mi].first, y = T.merges[mi].second;
      const int64_t ex = elems_of(info[x]), ey = elems_of(info[y]);
      const bool x_is_a = ex > ey || (ex == ey && info[x].wires.size() >= info[y].wires.size());
      const NodeInfo& A = info[x_is_a ? x : y];
      const NodeInfo& B = info[x_is_a ? y : x];
      NodeInfo C;
      StepDesc d;
      std::memset(&d, 0, sizeof(d));
      // node ids: leaves 0..L-1, the result of step j is L + j
      auto node_id = [&](int v) { return v < L ? v : L + step_of[v - L]; };
      d.a_node = node_id(x_is_a ? x : y);
      d.b_node = node_id(x_is_a ? y : x);
      d.c_node = L + (int)steps.size();
      step_of[mi] = (int)steps.size();
      std::vector<int> mw, kw, nw;
      for (int w : A.wires)
        (std::find(B.wires.begin(), B.wires.end(), w) != B.wires.end() ? kw : mw).push_back(w);
      for (int w : B.wires)
        if (std::find(A.wires.begin(), A.wires.end(), w) == A.wires.end()) nw.push_back(w);
      C.wires = node_order[L + mi];
      C.bmask = A.bmask | B.bmask;
      C.border = border_of[L + mi];
      if (C.wires.size() != mw.size() + nw.size() || (int)C.border.size() != __builtin_popcount(C.bmask))
        fail(TN_ERR_PLAN, "internal: layout of a step result");
      auto pos_in = [](const std::vector<int>& ws, int w) {
        return (int)(std::find(ws.begin(), ws.end(), w) - ws.begin());
      };
      // tile columns follow C's memory order (the epilogue's writes then run along C)
      std::stable_sort(nw.begin(), nw.end(), [&](int u, int v) { return pos_in(C.wires, u) < pos_in(C.wires, v); });
      // storage position of batch bit j in a node: rank + its index in the node's batch order
      auto bpos = [&](const NodeInfo& x, int j) { return (int)x.wires.size() + pos_in(x.border, j); };
      const int ra = (int)A.wires.size(), rb = (int)B.wires.size(), rc = (int)C.wires.size();
      std::vector<std::pair<int, int>> mb, nb;  // (pos in operand, pos in C)
      std::vector<std::array<int, 3>> bb;       // shared batch bits (pos A, pos B, pos C)
      for (int w : mw) mb.push_back({pos_in(A.wires, w), pos_in(C.wires, w)});
      for (int w : nw) nb.push_back({pos_in(B.wires, w), pos_in(C.wires, w)});
      for (int j : A.border) {   // rows: A's batch bits in A's storage order
        if ((B.bmask >> j) & 1) bb.push_back({bpos(A, j), bpos(B, j), bpos(C, j)});
        else mb.push_back({bpos(A, j), bpos(C, j)});
      }
      for (int j : B.border)
        if (!((A.bmask >> j) & 1)) nb.push_back({bpos(B, j), bpos(C, j)});
      if ((int)(mb.size() + kw.size()) > MAXR || (int)(kw.size() + nb.size()) > MAXR ||
          (int)(mb.size() + nb.size()) > MAXR || (int)bb.size() > MAXB)
        fail(TN_ERR_UNSUPPORTED, "a tensor exceeds the kernels' rank limit");
      d.nm = (int)mb.size();
      d.nk = (int)kw.size();
      d.nn = (int)nb.size();
      d.nb = (int)bb.size();
      d.nm_wires = (int)mw.size();
      d.nn_wires = (int)nw.size();
      d.rank_a = ra;
      d.rank_b = rb;
      d.rank_c = rc;
      for (int i = 0; i < d.nm; ++i) {
        d.a_mpos[i] = (int8_t)mb[i].first;
        d.c_mpos[i] = (int8_t)mb[i].second;
      }
      for (int i = 0; i < d.nk; ++i) {
        d.a_kpos[i] = (int8_t)pos_in(A.wires, kw[i]);
        d.b_kpos[i] = (int8_t)pos_in(B.wires, kw[i]);
      }
      for (int i = 0; i < d.nn; ++i) {
        d.b_npos[i] = (int8_t)nb[i].first;
        d.c_npos[i] = (int8_t)nb[i].second;
      }
      for (int i = 0; i < d.nb; ++i) {
        d.a_bpos[i] = (int8_t)bb[i][0];
        d.b_bpos[i] = (int8_t)bb[i][1];
        d.c_bpos[i] = (int8_t)bb[i][2];
      }
      d.a_elems = elems_of(A);
      d.b_elems = elems_of(B);
      d.a_off = A.off;
      d.b_off = B.off;
      if (pooled[L + mi] && C.bmask != 0) fail(TN_ERR_PLAN, "internal: pooled result with batch bits");
      C.off = pooled[L + mi] ? pool_off[L + mi] : alloc(elems_of(C));
      d.c_off = C.off;
      d.c_elems = elems_of(C);
      peak = std::max(peak, end);
      d.kernel = -1;
      d.group = exec_group[e];
      const int a_id = x_is_a ? x : y, b_id = x_is_a ? y : x;
      if (!pooled[a_id]) to_release.push_back({A.off, elems_of(A)});
      if (!pooled[b_id]) to_release.push_back({B.off, elems_of(B)});
      info[L + mi] = C;
      steps.push_back(d);
      if (exec_group[e] < 0 || e + 1 == exec.size() || exec_group[e + 1] != exec_group[e]) {
        for (auto [off, sz] : to_release) release(off, sz);
        to_release.clear();
      }
    }
    arena = peak;
    return peak * 8 <= cap_bytes;
  };

  std::vector<NodeInfo> info;
  std::vector<StepDesc> steps;
  std::vector<int> exec;   // merge index of every step, in execution order
  int64_t arena = 0;
  int b = o.log2_batch_slices > 0 ? std::min(o.log2_batch_slices, std::min(nS, 12)) : std::min(nS, 12);
  if (nF > 0) b = 0;   // caller-sliced plans contract one slice per chunk
  while (true) {
    const bool ok = layout(b, info, steps, arena, exec);
    if (ok) break;
    if (b == 0) fail(TN_ERR_PLAN, "one slice does not fit the arena cap");
    --b;
  }
  P->log2_batch = b;
  P->steps = steps;
  P->arena_elems = arena;
  // dependence of every step's result on the slice id (bit 0) and on the
  // closed output bits (bit 1): a step with neither computes the same tensor
  // in every chunk of every call
  for (size_t j = 0; j < P->steps.size(); ++j) P->steps[j].dep_flags = nflag[L + exec[j]];
  // the executor runs a group's steps concurrently: check that none reads
  // another's result and that no output overlaps another step's operands or output
  for (size_t i = 0; i < P->steps.size(); ++i) {
    const StepDesc& u = P->steps[i];
    if (u.group < 0) continue;
    for (size_t j = i + 1; j < P->steps.size() && P->steps[j].group == u.group; ++j) {
      const StepDesc& v = P->steps[j];
      auto overlap = [](int64_t o1, int64_t n1, int64_t o2, int64_t n2) { return o1 < o2 + n2 && o2 < o1 + n1; };
      if (v.a_node == u.c_node || v.b_node == u.c_node || u.a_node == v.c_node || u.b_node == v.c_node ||
          overlap(u.c_off, u.c_elems, v.a_off, v.a_elems) || overlap(u.c_off, u.c_elems, v.b_off, v.b_elems) ||
          overlap(v.c_off, v.c_elems, u.a_off, u.a_elems) || overlap(v.c_off, v.c_elems, u.b_off, u.b_elems) ||
          overlap(u.c_off, u.c_elems, v.c_off, v.c_elems) || u.dep_flags == 0 || v.dep_flags == 0 ||
          (u.dep_flags == 2) != (v.dep_flags == 2))   // one class: per batch (2) or per chunk (1, 3)
        fail(TN_ERR_PLAN, "internal: a step group is not independent");
    }
  }

  // leaves: source data ordered [kept planning wires, sliced wires by slice bit, closed outputs]
  P->leaves.resize(L);
  for (int i = 0; i < L; ++i) {
    const HTensor& lf = S.leaves[i];
    std::vector<int> ord, kind, idx;
    for (int w : info[i].wires) ord.push_back(wire_of_pw[w]);
    std::vector<std::pair<int, int>> sw;
    for (int w : lf.wires)
      if (!S.fixed[w] && SL.test(pw_of[w])) sw.push_back({slice_bit[pw_of[w]], w});
    std::sort(sw.begin(), sw.end());
    for (auto [j, w] : sw) {
      ord.push_back(w);
      kind.push_back(0);
      idx.push_back(j);
    }
    for (int w : lf.wires)
      if (S.fixed[w] && forced_bit[w] >= 0) {
        ord.push_back(w);
        kind.push_back(0);
        idx.push_back(forced_bit[w]);
      }
    for (int w : lf.wires)
      if (S.fixed[w] && forced_bit[w] < 0) {
        ord.push_back(w);
        kind.push_back(1);
        idx.push_back(net.labels[w].q);
      }
    if ((int)kind.size() > MAXFIX) fail(TN_ERR_UNSUPPORTED, "a leaf carries too many fixed wires");
    HTensor pt = hpermute(lf, ord);
    LeafDesc& ld = P->leaves[i];
    std::memset(&ld, 0, sizeof(ld));
    ld.src_off = (int64_t)P->leaf_data.size();
    ld.dst_off = info[i].off;
    ld.rank = (int)info[i].wires.size();
    ld.bmask = info[i].bmask;
    for (size_t t = 0; t < info[i].border.size(); ++t) ld.bslice[t] = (int8_t)info[i].border[t];
    ld.nfixed = (int)kind.size();
    for (size_t f = 0; f < kind.size(); ++f) {
      ld.fixed_kind[f] = (int8_t)kind[f];
      ld.fixed_index[f] = (int8_t)idx[f];
    }
    float am = 0.f;
    for (const cd& v : pt.data) {
      const std::complex<float> f((float)v.real(), (float)v.imag());
      P->leaf_data.push_back(f);
      am = std::max(am, std::max(std::fabs(f.real()), std::fabs(f.imag())));
    }
    P->leaf_amax.push_back(am);
  }
  // root
  const int root = (nm > 0) ? (L + order.back()) : 0;
  const NodeInfo& R = info[root];
  if ((int)R.wires.size() != k_open) fail(TN_ERR_PLAN, "internal: root rank differs from open qubits");
  P->root.off = R.off;
  P->root.rank = k_open;
  P->root.bmask = R.bmask;
  for (size_t t = 0; t < R.border.size(); ++t) P->root.bslice[t] = (int8_t)R.border[t];
  for (int j = 0; j < k_open; ++j) {
    const int w = pw_of[net.output_wire[P->open_qubits[j]]];
    const int p = (int)(std::find(R.wires.begin(), R.wires.end(), w) - R.wires.begin());
    if (p >= (int)R.wires.size()) fail(TN_ERR_PLAN, "internal: open wire missing from the root");
    P->root.pos_of_open[j] = (int8_t)p;
  }
  // statistics
  PlanStats& st = P->stats;
  for (int i = 0; i < L; ++i) st.log2_max = std::max(st.log2_max, (int)info[i].wires.size());
  for (const StepDesc& d : P->steps) {
    st.flops_slice += 8.0 * pow2(d.nm_wires + d.nk + d.nn_wires);
    st.bytes_slice += 8.0 * (pow2(d.rank_a) + pow2(d.rank_b) + pow2(d.rank_c));
    st.flops_chunk += 8.0 * pow2(d.nm + d.nk + d.nn + d.nb);
    st.bytes_chunk += 8.0 * (double)(d.a_elems + d.b_elems + d.c_elems);
    st.log2_max = std::max(st.log2_max, d.rank_c);
    st.khist[std::min(d.nk, 39)]++;
  }
  guard.release();
  return P;
}

}  // namespace tnx

using namespace tnx;

extern "C" tn_status tn_plan_default_opts(tn_plan_opts* o) {
  clear_error();
  if (!o) {
    set_error("tn_plan_default_opts: NULL");
    return TN_ERR_ARG;
  }
  std::memset(o, 0, sizeof(*o));
  o->open_mask = 0;
  o->max_log2_intermediate = 30;
  o->min_log2_slices = 0;
  o->seed = 1;
  o->trials = 64;
  o->precision = TN_PREC_FP32;
  o->complex_mult = 4;
  o->log2_batch_slices = 0;
  o->max_arena_bytes = (int64_t)96 << 30;
  o->mem_weight = 0.0;
  o->sm_pairs = 1;
  return TN_OK;
}

extern "C" tn_status tn_plan(const tn_network_t* net, const tn_plan_opts* opts, tn_plan_t** out) {
  try {
    clear_error();
    if (!net || !opts || !out) fail(TN_ERR_ARG, "tn_plan: NULL argument");
    *out = nullptr;
    if (!(opts->mem_weight <= 0.0 || (opts->mem_weight >= 1e-6 && opts->mem_weight <= 1e9)))
      fail(TN_ERR_ARG, "mem_weight must be <= 0 (default) or in [1e-6, 1e9]");
    if (opts->sm_pairs != 0 && opts->sm_pairs != 1) fail(TN_ERR_ARG, "sm_pairs must be 0 or 1");
    g_alpha = opts->mem_weight > 0.0 ? opts->mem_weight : 32.0;
    Plan* p = nullptr;
    try {
      p = build_plan(net->net, *opts);
    } catch (...) {
      g_alpha = 32.0;
      throw;
    }
    g_alpha = 32.0;
    auto* h = new (std::nothrow) tn_plan_s;
    if (!h) {
      delete p;
      fail(TN_ERR_OOM, "host allocation failed");
    }
    h->plan = std::move(*p);
    delete p;
    *out = h;
    return TN_OK;
  } catch (const TnError& e) {
    set_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return TN_ERR_OOM;
  }
}

extern "C" tn_status tn_plan_info(const tn_plan_t* h, tn_plan_stats* s) {
  clear_error();
  if (!h || !s) {
    set_error("tn_plan_info: NULL argument");
    return TN_ERR_ARG;
  }
  const Plan& p = h->plan;
  std::memset(s, 0, sizeof(*s));
  s->n_qubits = p.n_qubits;
  s->n_open = (int)p.open_qubits.size();
  s->n_leaves = p.n_leaves;
  s->n_steps = (int)p.steps.size();
  s->log2_slices = (int)p.sliced.size();
  s->log2_batch_slices = p.log2_batch;
  s->log2_max_intermediate = p.stats.log2_max;
  s->precision = p.opts.precision;
  s->flops_per_slice = p.stats.flops_slice;
  s->bytes_per_slice = p.stats.bytes_slice;
  s->flops_per_chunk = p.stats.flops_chunk;
  s->bytes_per_chunk = p.stats.bytes_chunk;
  s->arena_bytes = p.arena_elems * 8;
  for (int i = 0; i < 40; ++i) s->k_histogram[i] = p.stats.khist[i];
  s->complex_mult = p.opts.complex_mult;
  // steps that depend on the slice id run in every chunk (the others run once
  // per plan or per batch); one kernel each at least, plus leaf select, the
  // two slice-sum kernels and the chunk advance
  int per_chunk = 4;
  for (const StepDesc& d : p.steps) per_chunk += (d.dep_flags & 1) ? 1 : 0;
  s->n_kernel_launches_per_chunk = per_chunk;
  return TN_OK;
}

extern "C" tn_status tn_plan_sliced_wires(const tn_plan_t* h, int32_t* qubit, int32_t* t, int32_t cap,
                                          int32_t* count) {
  clear_error();
  if (!h || !count || (cap > 0 && (!qubit || !t))) {
    set_error("tn_plan_sliced_wires: NULL argument");
    return TN_ERR_ARG;
  }
  const Plan& p = h->plan;
  *count = (int)p.sliced.size();
  for (int j = 0; j < (int)p.sliced.size() && j < cap; ++j) {
    qubit[j] = p.sliced[j].q;
    t[j] = p.sliced[j].t;
  }
  return TN_OK;
}

extern "C" tn_status tn_plan_step_layout(const tn_plan_t* h, int32_t step, int32_t* out, int32_t cap,
                                         int32_t* count) {
  clear_error();
  if (!h || !out || !count) {
    set_error("tn_plan_step_layout: NULL argument");
    return TN_ERR_ARG;
  }
  const Plan& p = h->plan;
  if (step < 0 || step >= (int)p.steps.size()) {
    set_error("tn_plan_step_layout: step out of range");
    return TN_ERR_ARG;
  }
  const StepDesc& d = p.steps[step];
  std::vector<int32_t> v = {d.nm, d.nk, d.nn, d.nb};
  auto put = [&](const int8_t* pos, int n) {
    for (int i = 0; i < n; ++i) v.push_back(pos[i]);
  };
  put(d.a_mpos, d.nm);
  put(d.a_kpos, d.nk);
  put(d.b_kpos, d.nk);
  put(d.b_npos, d.nn);
  put(d.c_mpos, d.nm);
  put(d.c_npos, d.nn);
  put(d.a_bpos, d.nb);
  put(d.b_bpos, d.nb);
  put(d.c_bpos, d.nb);
  v.push_back(d.dep_flags);
  v.push_back(d.group);
  *count = (int32_t)v.size();
  if ((int32_t)v.size() > cap) {
    set_error("tn_plan_step_layout: cap smaller than the layout");
    return TN_ERR_ARG;
  }
  for (size_t i = 0; i < v.size(); ++i) out[i] = v[i];
  return TN_OK;
}

// Roofline time of one step over its batch instances: max(flops / peak,
// bytes / bandwidth), 8 flops per complex multiply-add, every operand read or
// written once as complex64.
static double step_model_seconds(const StepDesc& d, double peak_flops, double peak_bytes) {
  const double flops = 8.0 * std::ldexp(1.0, d.nm + d.nk + d.nn + d.nb);
  const double bytes = 8.0 * ((double)d.a_elems + (double)d.b_elems + (double)d.c_elems);
  return std::max(flops / peak_flops, bytes / peak_bytes);
}

extern "C" tn_status tn_plan_model_time(const tn_plan_t* h, double peak_flops, double peak_bytes,
                                        double* seconds) {
  clear_error();
  if (!h || !seconds) {
    set_error("tn_plan_model_time: NULL argument");
    return TN_ERR_ARG;
  }
  if (!(peak_flops > 0.0) || !(peak_bytes > 0.0) || !std::isfinite(peak_flops) || !std::isfinite(peak_bytes)) {
    set_error("tn_plan_model_time: peaks must be positive and finite");
    return TN_ERR_ARG;
  }
  double t = 0.0;
  for (const StepDesc& d : h->plan.steps)
    if (d.dep_flags & 1) t += step_model_seconds(d, peak_flops, peak_bytes);
  *seconds = t;
  return TN_OK;
}

extern "C" tn_status tn_plan_rank(const tn_network_t* net, const tn_plan_opts* opts, int32_t n_candidates,
                                  const uint64_t* seeds, const double* mem_weights, double peak_flops,
                                  double peak_bytes, double* model_seconds) {
  clear_error();
  if (!net || !opts || !seeds || !mem_weights || !model_seconds) {
    set_error("tn_plan_rank: NULL argument");
    return TN_ERR_ARG;
  }
  if (n_candidates < 1 || n_candidates > 100000) {
    set_error("tn_plan_rank: n_candidates must be in [1, 100000]");
    return TN_ERR_ARG;
  }
  if (!(peak_flops > 0.0) || !(peak_bytes > 0.0) || !std::isfinite(peak_flops) || !std::isfinite(peak_bytes)) {
    set_error("tn_plan_rank: peaks must be positive and finite");
    return TN_ERR_ARG;
  }
  for (int i = 0; i < n_candidates; ++i)
    if (!(mem_weights[i] <= 0.0 || (mem_weights[i] >= 1e-6 && mem_weights[i] <= 1e9))) {
      set_error("tn_plan_rank: mem_weight must be <= 0 (default) or in [1e-6, 1e9]");
      return TN_ERR_ARG;
    }
  int built = 0;
  for (int i = 0; i < n_candidates; ++i) {
    model_seconds[i] = -1.0;
    tn_plan_opts o = *opts;
    o.seed = seeds[i];
    o.mem_weight = mem_weights[i];
    tn_plan_t* h = nullptr;
    if (tn_plan(net, &o, &h) != TN_OK || !h) continue;   // e.g. no batch fits the arena cap
    double chunk = 0.0;
    if (tn_plan_model_time(h, peak_flops, peak_bytes, &chunk) == TN_OK) {
      // one batch: every chunk, plus the steps that run once per batch bitstring
      double per_batch = 0.0;
      for (const StepDesc& d : h->plan.steps)
        if (d.dep_flags == 2) per_batch += step_model_seconds(d, peak_flops, peak_bytes);
      model_seconds[i] = chunk * std::ldexp(1.0, (int)h->plan.sliced.size() - h->plan.log2_batch) + per_batch;
    }
    ++built;
    tn_plan_destroy(h);
  }
  clear_error();
  if (built == 0) {
    set_error("tn_plan_rank: no candidate plan could be built");
    return TN_ERR_PLAN;
  }
  return TN_OK;
}

extern "C" tn_status tn_plan_tree(const tn_plan_t* h, int32_t* leaf_of_gate, int32_t n_gates, int32_t* step_nodes,
                                  int32_t cap_steps, int32_t* n_leaves, int32_t* n_steps) {
  clear_error();
  if (!h || !leaf_of_gate || !step_nodes || !n_leaves || !n_steps) {
    set_error("tn_plan_tree: NULL argument");
    return TN_ERR_ARG;
  }
  const Plan& p = h->plan;
  int max_gate = -1;
  for (const auto& v : p.leaf_gates)
    for (int g : v) max_gate = std::max(max_gate, g);
  if (n_gates <= max_gate || n_gates < 0) {
    set_error("tn_plan_tree: n_gates is smaller than the circuit's gate count");
    return TN_ERR_ARG;
  }
  *n_leaves = (int32_t)p.leaf_gates.size();
  *n_steps = (int32_t)p.steps.size();
  if (cap_steps < (int32_t)p.steps.size()) {
    set_error("tn_plan_tree: cap_steps smaller than the plan's step count");
    return TN_ERR_ARG;
  }
  for (int g = 0; g < n_gates; ++g) leaf_of_gate[g] = -1;
  for (size_t l = 0; l < p.leaf_gates.size(); ++l)
    for (int g : p.leaf_gates[l]) leaf_of_gate[g] = (int32_t)l;
  for (size_t j = 0; j < p.steps.size(); ++j) {
    step_nodes[2 * j] = p.steps[j].a_node;
    step_nodes[2 * j + 1] = p.steps[j].b_node;
  }
  return TN_OK;
}

extern "C" tn_status tn_plan_step_shape(const tn_plan_t* h, int32_t step, int32_t* lm, int32_t* lk,
                                        int32_t* ln, int32_t* lb) {
  clear_error();
  if (!h || !lm || !lk || !ln || !lb) {
    set_error("tn_plan_step_shape: NULL argument");
    return TN_ERR_ARG;
  }
  const Plan& p = h->plan;
  if (step < 0 || step >= (int)p.steps.size()) {
    set_error("tn_plan_step_shape: step out of range");
    return TN_ERR_ARG;
  }
  const StepDesc& d = p.steps[step];
  *lm = d.nm;
  *lk = d.nk;
  *ln = d.nn;
  *lb = d.nb;
  return TN_OK;
}
