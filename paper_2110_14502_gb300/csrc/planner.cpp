// Contraction-order search, slicing, step layout and memory planning.
//
// Paper: Sec. "Searching for Better Contraction Paths with a Reduced
// Complexity" (the path decides the cost by orders of magnitude; the loss
// weighs complexity together with compute density) and Sec. "A PEPS-based
// Simulation Method with an Optimized Slicing Strategy" (slice S indices so
// each of the 2^S sub-networks fits in memory; the sub-networks are
// independent and their results are summed).
//
// Order search: many randomized trials of two generators -- a greedy pairwise
// merge with a noisy size score, and recursive bisection of the network graph
// refined with Fiduccia-Mattheyses moves -- each followed by greedy slicing.
// The trial with the smallest modelled GB300 time wins (the compute-density
// term: a step's time is the larger of its flops at the rate its kernel class
// reaches and its memory time; see step_time).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <random>
#include <tuple>

#include "tn_internal.h"

namespace tn {

namespace {

using LSet = std::vector<int>;  // sorted label ids

LSet sym_diff(const LSet& a, const LSet& b) {
  LSet r;
  std::set_symmetric_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(r));
  return r;
}
int union_size(const LSet& a, const LSet& b) {
  int i = 0, j = 0, n = 0;
  while (i < (int)a.size() && j < (int)b.size()) {
    if (a[i] == b[j]) { ++i; ++j; }
    else if (a[i] < b[j]) ++i;
    else ++j;
    ++n;
  }
  return n + (int)(a.size() - i) + (int)(b.size() - j);
}
int shared_count(const LSet& a, const LSet& b) {
  return (int)a.size() + (int)b.size() - union_size(a, b);
}
bool contains(const LSet& a, int l) { return std::binary_search(a.begin(), a.end(), l); }

// Modelled GB300 time of one step with operand widths wa, wb and wu = |A u B|:
// the larger of its flops at the rate of its kernel class and its memory
// time.  A tensor-core step reads its operands at HBM speed but writes its
// output through the epilogue's scattered per-thread stores, measured at
// about 3 TB/s; other steps move all their bytes at HBM speed.
double step_time(int wa, int wb, int wc, int wu) {
  const double flops = 8.0 * std::ldexp(1.0, wu);
  const double in = 8.0 * (std::ldexp(1.0, wa) + std::ldexp(1.0, wb)), out = 8.0 * std::ldexp(1.0, wc);
  int nk = (wa + wb - wc) / 2;
  int nm = wa - nk, nn = wb - nk;
  if (nm < nn) std::swap(nm, nn);
  const bool dense = nm >= 7 && nn >= 3 && nk >= 3;
  if (dense) return std::max(flops / 6.0e14, in / 6.0e12 + out / 3.0e12) + 1.5e-7;
  return std::max(flops / 6.0e13, (in + out) / 6.0e12) + 1.5e-7;
}

struct Builder {
  std::vector<LSet> sets;           // per SSA id
  std::vector<int> pairs;           // flattened SSA pairs
  explicit Builder(const std::vector<LSet>& leaves) : sets(leaves) {}
  int join(int a, int b) {
    sets.push_back(sym_diff(sets[a], sets[b]));
    pairs.push_back(a);
    pairs.push_back(b);
    return (int)sets.size() - 1;
  }
};

// Randomized greedy merge of the given ids (any SSA ids) into one root.
int greedy_join(Builder& B, std::vector<int> ids, double alpha, double tau, std::mt19937_64& rng) {
  if (ids.empty()) return -1;
  std::uniform_real_distribution<double> U(1e-12, 1.0);
  struct Cand { double s; int i, j; bool operator<(const Cand& o) const { return s > o.s; } };
  std::vector<char> alive;
  auto ensure = [&](int id) { if ((int)alive.size() <= id) alive.resize(id + 1, 0); };
  for (int id : ids) { ensure(id); alive[id] = 1; }
  // label -> active holders
  std::vector<std::vector<int>> holders;
  auto add_holder = [&](int id) {
    for (int l : B.sets[id]) {
      if ((int)holders.size() <= l) holders.resize(l + 1);
      holders[l].push_back(id);
    }
  };
  for (int id : ids) add_holder(id);
  auto score = [&](int i, int j) {
    const LSet &a = B.sets[i], &b = B.sets[j];
    int wc = (int)a.size() + (int)b.size() - 2 * shared_count(a, b);
    double s = std::log2(std::ldexp(1.0, wc)) - alpha * std::log2(std::ldexp(1.0, (int)a.size()) + std::ldexp(1.0, (int)b.size()));
    if (tau > 0) s -= tau * (-std::log(-std::log(U(rng))));
    return s;
  };
  std::vector<Cand> heap;
  auto push_pairs_of = [&](int id) {
    for (int l : B.sets[id]) {
      if (l >= (int)holders.size()) continue;
      for (int o : holders[l])
        if (o != id && alive[o]) {
          heap.push_back({score(std::min(o, id), std::max(o, id)), std::min(o, id), std::max(o, id)});
          std::push_heap(heap.begin(), heap.end());
        }
    }
  };
  for (int id : ids) push_pairs_of(id);
  int remaining = (int)ids.size();
  int last = ids[0];
  while (remaining > 1) {
    int i = -1, j = -1;
    while (!heap.empty()) {
      std::pop_heap(heap.begin(), heap.end());
      Cand c = heap.back();
      heap.pop_back();
      if (alive[c.i] && alive[c.j]) { i = c.i; j = c.j; break; }
    }
    if (i < 0) {  // disconnected: join the two smallest
      std::vector<int> act;
      for (int id = 0; id < (int)alive.size(); ++id)
        if (alive[id]) act.push_back(id);
      std::sort(act.begin(), act.end(), [&](int x, int y) {
        return B.sets[x].size() != B.sets[y].size() ? B.sets[x].size() < B.sets[y].size() : x < y;
      });
      i = act[0]; j = act[1];
    }
    alive[i] = alive[j] = 0;
    for (int l : B.sets[i]) { auto& h = holders[l]; h.erase(std::remove(h.begin(), h.end(), i), h.end()); }
    for (int l : B.sets[j]) { auto& h = holders[l]; h.erase(std::remove(h.begin(), h.end(), j), h.end()); }
    int nid = B.join(i, j);
    ensure(nid);
    alive[nid] = 1;
    add_holder(nid);
    push_pairs_of(nid);
    last = nid;
    --remaining;
  }
  return last;
}

// Fiduccia-Mattheyses bisection of `ids` (leaf-level SSA ids) minimising the
// number of shared labels cut, sizes within (1/2 +- eps).
void bisect(const Builder& B, const std::vector<int>& ids, double eps, std::mt19937_64& rng,
            std::vector<int>& part) {
  const int n = (int)ids.size();
  // adjacency via labels
  std::vector<std::vector<std::pair<int, int>>> adj(n);
  {
    std::vector<std::pair<int, int>> lab;  // (label, local idx)
    for (int v = 0; v < n; ++v)
      for (int l : B.sets[ids[v]]) lab.push_back({l, v});
    std::sort(lab.begin(), lab.end());
    std::vector<std::vector<int>> w(0);
    for (size_t s = 0; s < lab.size();) {
      size_t e = s;
      while (e < lab.size() && lab[e].first == lab[s].first) ++e;
      for (size_t x = s; x < e; ++x)
        for (size_t y = x + 1; y < e; ++y) {
          adj[lab[x].second].push_back({lab[y].second, 1});
          adj[lab[y].second].push_back({lab[x].second, 1});
        }
      s = e;
    }
    for (auto& a : adj) {  // merge parallel edges
      std::sort(a.begin(), a.end());
      std::vector<std::pair<int, int>> m;
      for (auto& p : a) {
        if (!m.empty() && m.back().first == p.first) m.back().second += p.second;
        else m.push_back(p);
      }
      a.swap(m);
    }
  }
  const int lo = std::max(1, (int)std::floor(n * (0.5 - eps)));
  const int hi = std::min(n - 1, (int)std::ceil(n * (0.5 + eps)));
  // initial: BFS growth from a random vertex up to a random target size
  part.assign(n, 1);
  std::uniform_int_distribution<int> pick(0, n - 1);
  int target = std::uniform_int_distribution<int>(lo, hi)(rng);
  {
    std::vector<int> q;
    std::vector<char> seen(n, 0);
    int count = 0;
    int start = pick(rng);
    q.push_back(start);
    seen[start] = 1;
    size_t head = 0;
    while (count < target) {
      if (head == q.size()) {
        int v;
        do v = pick(rng); while (seen[v]);
        seen[v] = 1;
        q.push_back(v);
      }
      int v = q[head++];
      part[v] = 0;
      ++count;
      for (auto& e : adj[v])
        if (!seen[e.first]) { seen[e.first] = 1; q.push_back(e.first); }
    }
  }
  auto gain_of = [&](int v) {
    int g = 0;
    for (auto& e : adj[v]) g += (part[e.first] != part[v]) ? e.second : -e.second;
    return g;
  };
  int size0 = 0;
  for (int v = 0; v < n; ++v) size0 += part[v] == 0;
  for (int pass = 0; pass < 10; ++pass) {
    std::vector<char> locked(n, 0);
    std::vector<int> gain(n);
    for (int v = 0; v < n; ++v) gain[v] = gain_of(v);
    std::vector<int> moves;
    int cur = 0, best = 0, best_len = 0, s0 = size0;
    for (int step = 0; step < n; ++step) {
      int bv = -1, bg = -(1 << 30);
      for (int v = 0; v < n; ++v) {
        if (locked[v]) continue;
        int ns0 = s0 + (part[v] == 0 ? -1 : 1);
        if (ns0 < lo || ns0 > hi) continue;
        if (gain[v] > bg) { bg = gain[v]; bv = v; }
      }
      if (bv < 0) break;
      locked[bv] = 1;
      s0 += part[bv] == 0 ? -1 : 1;
      part[bv] ^= 1;
      cur += bg;
      moves.push_back(bv);
      gain[bv] = -gain[bv];
      for (auto& e : adj[bv]) {
        int u = e.first;
        gain[u] += (part[u] == part[bv]) ? -2 * e.second : 2 * e.second;
      }
      if (cur > best) { best = cur; best_len = (int)moves.size(); }
    }
    for (int k = (int)moves.size() - 1; k >= best_len; --k) part[moves[k]] ^= 1;
    size0 = 0;
    for (int v = 0; v < n; ++v) size0 += part[v] == 0;
    if (best <= 0) break;
  }
}

int bisect_tree(Builder& B, const std::vector<int>& ids, int cutoff, double eps, double alpha,
                std::mt19937_64& rng) {
  if ((int)ids.size() <= cutoff) return greedy_join(B, ids, alpha, 0.0, rng);
  std::vector<int> part;
  bisect(B, ids, eps, rng, part);
  std::vector<int> s0, s1;
  for (size_t v = 0; v < ids.size(); ++v) (part[v] ? s1 : s0).push_back(ids[v]);
  if (s0.empty() || s1.empty()) return greedy_join(B, ids, alpha, 0.0, rng);
  int a = bisect_tree(B, s0, cutoff, eps, alpha, rng);
  int b = bisect_tree(B, s1, cutoff, eps, alpha, rng);
  return B.join(a, b);
}

// PEPS-style lattice order (Sec. "A PEPS-based Simulation Method with an
// Optimized Slicing Strategy"): a leaf sits at the grid site of the lowest
// qubit among its wires and at the earliest time step; the leaves of every
// grid column (or row) are merged one after another in (row, time) order into
// one boundary tensor of that line, and the lines are then absorbed one by one
// from one side of the grid to the other.  variant: bit 0 sweeps rows instead
// of columns, bit 1 starts from the far side.
int lattice_join(Builder& B, const Network& net, int variant) {
  const int L = (int)net.leaves.size();
  const int cols = net.cols > 0 ? net.cols : std::max(net.n, 1);
  std::vector<std::tuple<int, int, int, int>> key;  // (line, position along it, time, leaf)
  for (int i = 0; i < L; ++i) {
    int q = net.n, t = 1 << 30;
    for (int l : net.leaves[i].labels) {
      if (net.wire[l].first < 0) continue;  // bond of a split diagonal: no grid site
      q = std::min(q, net.wire[l].first);
      t = std::min(t, net.wire[l].second);
    }
    if (q >= net.n) q = 0;
    const int r = q / cols, c = q % cols;
    int line = (variant & 1) ? r : c, pos = (variant & 1) ? c : r;
    if (variant & 2) line = -line;
    key.emplace_back(line, pos, t, i);
  }
  std::sort(key.begin(), key.end());
  int acc = -1;
  for (size_t i = 0; i < key.size();) {
    int col = -1;
    size_t j = i;
    for (; j < key.size() && std::get<0>(key[j]) == std::get<0>(key[i]); ++j)
      col = col < 0 ? std::get<3>(key[j]) : B.join(col, std::get<3>(key[j]));
    acc = acc < 0 ? col : B.join(acc, col);
    i = j;
  }
  return acc;
}

struct Eval {
  double time = 0, cmac = 0;
  int width = 0;
  std::vector<int> sliced;
};

// Node label sets of a tree (leaf sets given), with the sliced labels removed.
void node_sets(const std::vector<LSet>& leaves, const std::vector<int>& pairs,
               const std::vector<int>& sliced, std::vector<LSet>& sets) {
  sets.clear();
  for (auto& s : leaves) {
    LSet t;
    for (int l : s)
      if (std::find(sliced.begin(), sliced.end(), l) == sliced.end()) t.push_back(l);
    sets.push_back(t);
  }
  for (size_t p = 0; p < pairs.size(); p += 2) sets.push_back(sym_diff(sets[pairs[p]], sets[pairs[p + 1]]));
}

// Weight of every step of a tree in the modelled time: `hint` for a step whose
// subtree holds a bitstring-dependent leaf (it runs once per bitstring and
// slice), 1 for the others (once per slice, shared by the bitstrings).
std::vector<double> step_weights(const std::vector<char>& var_leaf, const std::vector<int>& pairs, double hint) {
  std::vector<char> var(var_leaf);
  std::vector<double> w(pairs.size() / 2);
  for (size_t p = 0; p < pairs.size(); p += 2) {
    const char v = var[pairs[p]] | var[pairs[p + 1]];
    var.push_back(v);
    w[p / 2] = v ? hint : 1.0;
  }
  return w;
}

void cost_of(const std::vector<LSet>& sets, const std::vector<int>& pairs, int L, const std::vector<double>& w,
             double& time, double& cmac, int& width) {
  time = 0; cmac = 0; width = 0;
  for (auto& s : sets) width = std::max(width, (int)s.size());
  for (size_t p = 0; p < pairs.size(); p += 2) {
    const LSet &a = sets[pairs[p]], &b = sets[pairs[p + 1]], &c = sets[L + p / 2];
    int wu = union_size(a, b);
    cmac += std::ldexp(1.0, wu);
    time += w[p / 2] * step_time((int)a.size(), (int)b.size(), (int)c.size(), wu);
  }
}

// Greedy slicing: repeatedly remove the label (present in a widest node) that
// gives the smallest (width, modelled time).  Removing a label only changes
// the steps and nodes that hold it, so each candidate is scored incrementally.
Eval slice_tree(const std::vector<LSet>& leaves, const std::vector<int>& pairs, const LSet& sliceable,
                int num_sliced, int cap, const std::vector<double>& wt) {
  const int L = (int)leaves.size();
  const int nsteps = (int)pairs.size() / 2;
  Eval ev;
  std::vector<LSet> sets;
  node_sets(leaves, pairs, ev.sliced, sets);
  // per step widths, per node sizes, and where every label occurs
  std::vector<int> wa(nsteps), wb(nsteps), wc(nsteps), wu(nsteps);
  std::vector<int> size(sets.size());
  int maxlab = 0;
  for (auto& st : sets)
    for (int l : st) maxlab = std::max(maxlab, l + 1);
  std::vector<std::vector<int>> in_node(maxlab), in_step(maxlab);
  for (size_t v = 0; v < sets.size(); ++v) {
    size[v] = (int)sets[v].size();
    for (int l : sets[v]) in_node[l].push_back((int)v);
  }
  for (int t = 0; t < nsteps; ++t) {
    const LSet &a = sets[pairs[2 * t]], &b = sets[pairs[2 * t + 1]];
    wa[t] = (int)a.size();
    wb[t] = (int)b.size();
    wc[t] = (int)sets[L + t].size();
    wu[t] = union_size(a, b);
    LSet u;
    std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(u));
    for (int l : u) in_step[l].push_back(t);
  }
  std::vector<char> removed(maxlab, 0);
  auto totals = [&](double& time, double& cmac, int& width) {
    time = 0; cmac = 0; width = 0;
    for (int v : size) width = std::max(width, v);
    for (int t = 0; t < nsteps; ++t) {
      cmac += std::ldexp(1.0, wu[t]);
      time += wt[t] * step_time(wa[t], wb[t], wc[t], wu[t]);
    }
  };
  totals(ev.time, ev.cmac, ev.width);
  auto need_more = [&]() {
    if (num_sliced >= 0) return (int)ev.sliced.size() < num_sliced;
    return cap > 0 && ev.width > cap;
  };
  while (need_more()) {
    // width histogram to update the maximum after a removal
    std::vector<int> hist(ev.width + 2, 0);
    for (int v : size) hist[v]++;
    LSet cand;
    for (size_t v = 0; v < sets.size(); ++v)
      if (size[v] == ev.width)
        for (int l : sets[v])
          if (!removed[l] && contains(sliceable, l)) cand.push_back(l);
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    if (cand.empty()) {  // widest nodes hold only open labels: slice elsewhere
      for (int l = 0; l < maxlab; ++l)
        if (!removed[l] && !in_node[l].empty() && contains(sliceable, l)) cand.push_back(l);
    }
    if (cand.empty()) break;
    int best = -1, bw = 0;
    double bt = 0;
    for (int l : cand) {
      // new maximum width: nodes holding l shrink by one
      int at_max = hist[ev.width], holding_max = 0;
      for (int v : in_node[l]) holding_max += size[v] == ev.width;
      const int w = (at_max > holding_max) ? ev.width : ev.width - 1;
      double dt = 0;
      for (int t : in_step[l]) {
        const int a_has = std::binary_search(sets[pairs[2 * t]].begin(), sets[pairs[2 * t]].end(), l);
        const int b_has = std::binary_search(sets[pairs[2 * t + 1]].begin(), sets[pairs[2 * t + 1]].end(), l);
        const int c_has = a_has != b_has;
        dt += wt[t] * (step_time(wa[t] - a_has, wb[t] - b_has, wc[t] - c_has, wu[t] - 1) -
                       step_time(wa[t], wb[t], wc[t], wu[t]));
      }
      const double t_new = ev.time + dt;
      if (best < 0 || w < bw || (w == bw && t_new < bt)) { best = l; bw = w; bt = t_new; }
    }
    // apply the removal
    for (int t : in_step[best]) {
      const int a_has = std::binary_search(sets[pairs[2 * t]].begin(), sets[pairs[2 * t]].end(), best);
      const int b_has = std::binary_search(sets[pairs[2 * t + 1]].begin(), sets[pairs[2 * t + 1]].end(), best);
      wa[t] -= a_has;
      wb[t] -= b_has;
      wc[t] -= a_has != b_has;
      wu[t] -= 1;
    }
    for (int v : in_node[best]) {
      size[v] -= 1;
      auto& st = sets[v];
      st.erase(std::lower_bound(st.begin(), st.end(), best));
    }
    in_node[best].clear();
    in_step[best].clear();
    removed[best] = 1;
    ev.sliced.push_back(best);
    totals(ev.time, ev.cmac, ev.width);
  }
  return ev;
}

// Subtree reconfiguration: for each internal node, expand its subtree into a
// frontier of up to `k` sub-tensors (largest first) and replace the part
// above the frontier by the exact optimum over all contraction orders of the
// frontier (dynamic programming over subsets), under the step-time model.
// The frontier's joint label set is order independent, so every rewrite keeps
// the tree valid.  With wcap > 0 no new intermediate may hold more than wcap
// unsliced labels, so a rewrite never breaks the per-slice width cap.
void reconfigure(const std::vector<LSet>& leaves, std::vector<int>& pairs, const std::vector<int>& sliced,
                 int k, int passes, const std::vector<char>& var_leaf, double hint, int wcap) {
  const int L = (int)leaves.size();
  if (L < 3) return;
  std::vector<int> lch(L, -1), rch(L, -1);
  for (size_t p = 0; p < pairs.size(); p += 2) { lch.push_back(pairs[p]); rch.push_back(pairs[p + 1]); }
  int root = (int)lch.size() - 1;
  std::vector<LSet> sets;
  node_sets(leaves, pairs, sliced, sets);
  // bitstring dependence of every node (weight `hint` on the steps that have it)
  std::vector<char> var(var_leaf);
  for (size_t p = 0; p < pairs.size(); p += 2) var.push_back(var[pairs[p]] | var[pairs[p + 1]]);
  auto cost2 = [&](const LSet& a, const LSet& b, bool v) {
    int u = union_size(a, b);
    int sh = (int)a.size() + (int)b.size() - u;
    return (v ? hint : 1.0) * step_time((int)a.size(), (int)b.size(), u - sh, u);
  };
  for (int pass = 0; pass < passes; ++pass) {
    // post-order list of internal nodes reachable from the root
    std::vector<int> post, stack{root};
    std::vector<int> tmp;
    while (!stack.empty()) {
      int v = stack.back(); stack.pop_back();
      if (lch[v] < 0) continue;
      tmp.push_back(v);
      stack.push_back(lch[v]);
      stack.push_back(rch[v]);
    }
    post.assign(tmp.rbegin(), tmp.rend());
    bool improved = false;
    for (int v : post) {
      std::vector<int> front{lch[v], rch[v]};
      std::vector<int> expanded{v};
      while ((int)front.size() < k) {
        int bi = -1;
        for (int i = 0; i < (int)front.size(); ++i)
          if (lch[front[i]] >= 0 && (bi < 0 || sets[front[i]].size() > sets[front[bi]].size())) bi = i;
        if (bi < 0) break;
        int u = front[bi];
        expanded.push_back(u);
        front[bi] = lch[u];
        front.push_back(rch[u]);
      }
      const int f = (int)front.size();
      if (f < 3) continue;
      double cur = 0;
      for (int u : expanded) cur += cost2(sets[lch[u]], sets[rch[u]], var[u]);
      const int full = (1 << f) - 1;
      std::vector<LSet> ss(1 << f);
      std::vector<char> vs(1 << f, 0);
      std::vector<double> best(1 << f, 0.0);
      std::vector<int> split(1 << f, 0);
      for (int S = 1; S <= full; ++S) {
        int low = S & -S;
        if (S == low) { ss[S] = sets[front[__builtin_ctz(S)]]; vs[S] = var[front[__builtin_ctz(S)]]; continue; }
        ss[S] = sym_diff(ss[S ^ low], ss[low]);
        vs[S] = vs[S ^ low] | vs[low];
        if (wcap > 0 && S != full && (int)ss[S].size() > wcap) {  // over the width cap: never built
          best[S] = 1e300;
          continue;
        }
        double b = 1e300;
        int bs = 0;
        // sub-splits containing the lowest bit
        for (int S1 = (S - 1) & S; S1 > 0; S1 = (S1 - 1) & S) {
          if (!(S1 & low)) continue;
          int S2 = S ^ S1;
          double c = best[S1] + best[S2] + cost2(ss[S1], ss[S2], vs[S]);
          if (c < b) { b = c; bs = S1; }
        }
        best[S] = b;
        split[S] = bs;
      }
      if (best[full] < cur * (1 - 1e-9) - 1e-12) {
        // rebuild: v keeps its id as the root of the rewritten part
        std::function<int(int)> build = [&](int S) -> int {
          if ((S & (S - 1)) == 0) return front[__builtin_ctz(S)];
          int a = build(split[S]), b = build(S ^ split[S]);
          lch.push_back(a); rch.push_back(b);
          sets.push_back(sym_diff(sets[a], sets[b]));
          var.push_back(var[a] | var[b]);
          return (int)lch.size() - 1;
        };
        int a = build(split[full]), b = build(full ^ split[full]);
        lch[v] = a; rch[v] = b;
        improved = true;
      }
    }
    if (!improved) break;
  }
  // re-emit SSA pairs in post-order
  std::vector<int> id(lch.size(), -1);
  for (int i = 0; i < L; ++i) id[i] = i;
  std::vector<int> out;
  int nid = L;
  std::vector<std::pair<int, int>> st{{root, 0}};
  while (!st.empty()) {
    auto& [v, state] = st.back();
    if (lch[v] < 0) { st.pop_back(); continue; }
    if (state == 0) { state = 1; st.push_back({lch[v], 0}); continue; }
    if (state == 1) { state = 2; st.push_back({rch[v], 0}); continue; }
    out.push_back(id[lch[v]]);
    out.push_back(id[rch[v]]);
    id[v] = nid++;
    st.pop_back();
  }
  pairs.swap(out);
}

void put32(std::vector<uint8_t>& b, int32_t v) {
  uint8_t t[4];
  std::memcpy(t, &v, 4);
  b.insert(b.end(), t, t + 4);
}

uint64_t fnv1a(const std::vector<uint8_t>& b) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (uint8_t x : b) { h ^= x; h *= 0x100000001b3ull; }
  return h;
}

}  // namespace

tn_status make_plan(const Network& net, const tn_plan_opts& opts, Plan& P) {
  P.net = net;
  P.opts = opts;
  const int L = (int)net.leaves.size();
  if (L == 0) return fail(TN_EINVAL, "tn_plan: empty network");
  std::vector<LSet> leaves(L);
  LSet sliceable;
  // leaves holding a closed output index depend on the bitstring
  std::vector<char> var_leaf(L, 0);
  const double hint = std::max(1, opts.bitstrings_hint);
  for (int i = 0; i < L; ++i) {
    for (int l : net.leaves[i].labels)
      if (net.kind[l] != LK_CLOSED) leaves[i].push_back(l);
      else var_leaf[i] = 1;
    std::sort(leaves[i].begin(), leaves[i].end());
    for (int l : leaves[i])
      if (net.kind[l] == LK_INTERNAL) sliceable.push_back(l);
  }
  std::sort(sliceable.begin(), sliceable.end());
  sliceable.erase(std::unique(sliceable.begin(), sliceable.end()), sliceable.end());
  if (opts.num_sliced > (int)sliceable.size())
    return fail(TN_EINVAL, "tn_plan: num_sliced %d exceeds the %d internal indices", opts.num_sliced,
                (int)sliceable.size());

  const int trials = opts.search_trials > 0 ? opts.search_trials : 128;
  std::vector<int> all(L);
  std::iota(all.begin(), all.end(), 0);
  // One search: `trials` randomized trees, each sliced and rewritten, the best
  // kept and polished.  With cap_aware the rewrites after slicing build no
  // intermediate wider than the width cap; otherwise they may, and a trial
  // whose rewrite broke the cap only wins when no trial kept it.
  auto search = [&](bool cap_aware, Eval& best, std::vector<int>& best_pairs) -> bool {
    const int wcap = cap_aware ? opts.max_log2_intermediate : 0;
    std::mt19937_64 rng(opts.seed ^ 0x5DEECE66Dull);
    bool have = false;
    for (int t = 0; t < (L == 1 ? 1 : trials); ++t) {
      Builder B(leaves);
      std::mt19937_64 r2(rng());
      if (L > 1 && opts.order_generator == 1) {
        lattice_join(B, net, t % 4);
      } else if (L > 1) {
        if (t % 2 == 0) {
          double alpha = std::uniform_real_distribution<double>(0.0, 1.5)(r2);
          const double taus[] = {0.0, 0.01, 0.05, 0.1, 0.3, 1.0};
          double tau = taus[std::uniform_int_distribution<int>(0, 5)(r2)];
          greedy_join(B, all, alpha, tau, r2);
        } else {
          int cutoff = std::uniform_int_distribution<int>(4, 24)(r2);
          double eps = std::uniform_real_distribution<double>(0.02, 0.4)(r2);
          double alpha = std::uniform_real_distribution<double>(0.0, 1.0)(r2);
          bisect_tree(B, all, cutoff, eps, alpha, r2);
        }
      }
      reconfigure(leaves, B.pairs, {}, 6, 3, var_leaf, hint, 0);
      if (opts.max_log2_cmac > 0) {
        // slicing only adds work: a tree already above the cost cap is dropped unsliced
        std::vector<LSet> st0;
        node_sets(leaves, B.pairs, {}, st0);
        double t0, c0;
        int w0;
        cost_of(st0, B.pairs, L, step_weights(var_leaf, B.pairs, hint), t0, c0, w0);
        if (std::log2(std::max(c0, 1.0)) > opts.max_log2_cmac) continue;
      }
      Eval ev = slice_tree(leaves, B.pairs, sliceable, opts.num_sliced, opts.max_log2_intermediate,
                           step_weights(var_leaf, B.pairs, hint));
      if (!ev.sliced.empty()) {
        reconfigure(leaves, B.pairs, ev.sliced, 6, 3, var_leaf, hint, wcap);
        std::vector<LSet> st;
        node_sets(leaves, B.pairs, ev.sliced, st);
        cost_of(st, B.pairs, L, step_weights(var_leaf, B.pairs, hint), ev.time, ev.cmac, ev.width);
      }
      double score = ev.time * std::ldexp(1.0, (int)ev.sliced.size());
      double bscore = have ? best.time * std::ldexp(1.0, (int)best.sliced.size()) : 0;
      bool ok_cap = opts.max_log2_intermediate <= 0 || ev.width <= opts.max_log2_intermediate;
      bool bok_cap = have && (opts.max_log2_intermediate <= 0 || best.width <= opts.max_log2_intermediate);
      if (!have || (ok_cap && !bok_cap) || (ok_cap == bok_cap && score < bscore)) {
        best = ev;
        best_pairs = B.pairs;
        have = true;
      }
    }
    if (have && L > 2) {  // polish the winner with a wider window
      reconfigure(leaves, best_pairs, best.sliced, 8, 6, var_leaf, hint, wcap);
      std::vector<LSet> st;
      node_sets(leaves, best_pairs, best.sliced, st);
      cost_of(st, best_pairs, L, step_weights(var_leaf, best_pairs, hint), best.time, best.cmac, best.width);
    }
    return have;
  };
  Eval best;
  std::vector<int> best_pairs;
  const bool cap_aware = opts.cap_aware_rewrites == 1;
  bool have = search(cap_aware, best, best_pairs);
  if (have && !cap_aware && opts.max_log2_intermediate > 0 && best.width > opts.max_log2_intermediate) {
    // every trial's rewrites broke the width cap: search again keeping it
    Eval b2;
    std::vector<int> p2;
    if (search(true, b2, p2)) {
      best = b2;
      best_pairs.swap(p2);
    }
  }
  if (!have)
    return fail(TN_ETOOBIG, "tn_plan: every searched order costs more than the cap 2^%.1f CMAC", opts.max_log2_cmac);
  if (opts.max_log2_intermediate > 0 && best.width > opts.max_log2_intermediate)
    return fail(TN_ETOOBIG, "tn_plan: could not reach width 2^%d (best 2^%d with %d sliced)",
                opts.max_log2_intermediate, best.width, (int)best.sliced.size());
  if (best.width > 30)
    return fail(TN_ETOOBIG, "tn_plan: per-slice width 2^%d (cost 2^%.1f CMAC per slice) exceeds the 2^30 element limit; slice more",
                best.width, std::log2(std::max(best.cmac, 1.0)));
  double log2_total = std::log2(std::max(best.cmac, 1.0)) + (double)best.sliced.size();
  if (opts.max_log2_cmac > 0 && log2_total > opts.max_log2_cmac)
    return fail(TN_ETOOBIG, "tn_plan: cost 2^%.1f CMAC exceeds the cap 2^%.1f", log2_total, opts.max_log2_cmac);

  P.sliced = best.sliced;
  P.tree = best_pairs;
  P.cmac_per_slice = best.cmac;
  P.max_width = best.width;

  // ---- leaves: fixed indices and sub-labels; dependence (bit 0 closed, bit 1 sliced)
  std::vector<int> slice_bit(net.num_labels(), -1);
  for (size_t j = 0; j < P.sliced.size(); ++j) slice_bit[P.sliced[j]] = (int)j;
  P.leaf_use.assign(L, LeafUse());
  std::vector<int> dep(L + best_pairs.size() / 2, 0);
  int64_t store = 0;
  for (int i = 0; i < L; ++i) {
    LeafUse& U = P.leaf_use[i];
    const Leaf& lf = net.leaves[i];
    U.store_off = store;
    store += ((int64_t(1) << lf.labels.size()) + 31) & ~int64_t(31);  // 256-byte aligned leaves
    for (int l : lf.labels) {
      if (net.kind[l] == LK_CLOSED) { U.fixed_src.push_back(-2 - net.closed_qubit[l]); dep[i] |= 1; }
      else if (slice_bit[l] >= 0) { U.fixed_src.push_back(slice_bit[l]); dep[i] |= 2; }
      else { U.fixed_src.push_back(-1); U.sub_labels.push_back(l); }
    }
    U.variant = dep[i] != 0;
    U.phase = dep[i] == 0 ? 0 : dep[i] == 2 ? 1 : 2;
  }
  P.leaf_store_elems = store;

  // ---- steps (tree order); phase 0 invariant, 1 slice-only, 2 per (bitstring, slice)
  std::vector<LSet> order(L);  // memory label order of each SSA id
  for (int i = 0; i < L; ++i) order[i] = P.leaf_use[i].sub_labels;
  P.steps.clear();
  P.cmac_slice_only = 0;
  for (size_t p = 0; p < best_pairs.size(); p += 2) {
    int x = best_pairs[p], y = best_pairs[p + 1];
    Step S;
    const LSet &ox = order[x], &oy = order[y];
    bool swap = oy.size() > ox.size();
    S.a = swap ? y : x;
    S.b = swap ? x : y;
    S.la = order[S.a];
    S.lb = order[S.b];
    for (int l : S.la)
      if (std::find(S.lb.begin(), S.lb.end(), l) == S.lb.end()) S.lc.push_back(l);
    for (int l : S.lb)
      if (std::find(S.la.begin(), S.la.end(), l) == S.la.end()) S.lc.push_back(l);
    S.nk = (int)(S.la.size() + S.lb.size() - S.lc.size()) / 2;
    S.nm = (int)S.la.size() - S.nk;
    S.nn = (int)S.lb.size() - S.nk;
    // bandwidth-bound streaming kernel: N <= 16 with K <= 16, or N <= 8 with K <= 128
    S.klass = ((S.nn <= 4 && S.nk <= 4) || (S.nn <= 3 && S.nk <= 7)) ? SC_VECTOR : SC_SIMT;
    int d = dep[S.a] | dep[S.b];
    dep[L + p / 2] = d;
    S.variant = d != 0;
    S.phase = d == 0 ? 0 : d == 2 ? 1 : 2;
    if (S.phase == 1) P.cmac_slice_only += std::ldexp(1.0, S.nm + S.nn + S.nk);
    order.push_back(S.lc);
    P.steps.push_back(S);
  }
  auto phase_of = [&](int id) { return id < L ? P.leaf_use[id].phase : P.steps[id - L].phase; };

  // ---- output layouts, decided from the root down: every intermediate is
  // written with the indices its consumer contracts innermost (in one order
  // shared by both operands of the consumer), so the consumer's GEMM reads
  // contiguous K runs from both operands -- the permutation of the next step
  // is folded into this step's epilogue.
  {
    // label sets of every SSA id (order-free) to tell a step's two sides apart
    std::vector<LSet> sets(L + P.steps.size());
    for (int i = 0; i < L; ++i) { sets[i] = order[i]; std::sort(sets[i].begin(), sets[i].end()); }
    for (size_t s = 0; s < P.steps.size(); ++s) {
      sets[L + s] = P.steps[s].lc;
      std::sort(sets[L + s].begin(), sets[L + s].end());
    }
    for (int t = (int)P.steps.size() - 1; t >= 0; --t) {
      Step& S = P.steps[t];
      const LSet& ct = order[L + t];  // final layout of this step's output
      LSet kt;
      const int leaf_op = S.a < L ? S.a : (S.b < L ? S.b : -1);
      if (leaf_op >= 0) {
        // a leaf keeps its layout: the contracted indices follow its order
        const LSet& other = leaf_op == S.a ? order[S.b] : order[S.a];
        for (int l : order[leaf_op])
          if (std::find(other.begin(), other.end(), l) != other.end()) kt.push_back(l);
      } else {
        // contracted indices, innermost the ones that come from the larger side
        // of the larger operand's producer (its epilogue then writes one run)
        const int p = S.a - L;
        const LSet& sa = sets[P.steps[p].a];
        LSet from_a, from_b;
        for (int l : order[S.a])
          if (std::binary_search(sets[S.b].begin(), sets[S.b].end(), l))
            (std::binary_search(sa.begin(), sa.end(), l) ? from_a : from_b).push_back(l);
        if (from_a.size() >= from_b.size()) { kt = from_b; kt.insert(kt.end(), from_a.begin(), from_a.end()); }
        else { kt = from_a; kt.insert(kt.end(), from_b.begin(), from_b.end()); }
      }
      for (int x : {S.a, S.b}) {
        if (x < L) continue;
        // free indices in the order they take in this step's output, so the
        // GEMM's row / column bits follow the output's memory order
        LSet nl;
        for (int l : ct)
          if (std::binary_search(sets[x].begin(), sets[x].end(), l)) nl.push_back(l);
        nl.insert(nl.end(), kt.begin(), kt.end());
        order[x] = nl;
        P.steps[x - L].lc = nl;
      }
    }
    for (auto& S : P.steps) {
      S.la = order[S.a];
      S.lb = order[S.b];
    }
  }

  // ---- memory: invariant store (no reuse), slice arena and pair arena (first-fit with liveness)
  auto align = [](int64_t v) { return (v + 31) & ~int64_t(31); };
  struct Blk { int64_t off, size; };
  struct Arena {
    std::vector<Blk> freel;
    int64_t top = 0, peak = 0;
  } ar[3];
  auto alloc = [&](Arena& A, int64_t sz) {
    sz = align(sz);
    for (size_t i = 0; i < A.freel.size(); ++i)
      if (A.freel[i].size >= sz) {
        int64_t o = A.freel[i].off;
        A.freel[i].off += sz;
        A.freel[i].size -= sz;
        if (A.freel[i].size == 0) A.freel.erase(A.freel.begin() + i);
        return o;
      }
    int64_t o = A.top;
    A.top += sz;
    A.peak = std::max(A.peak, A.top);
    return o;
  };
  auto release = [&](Arena& A, int64_t off, int64_t sz) {
    sz = align(sz);
    A.freel.push_back({off, sz});
    std::sort(A.freel.begin(), A.freel.end(), [](const Blk& a, const Blk& b) { return a.off < b.off; });
    std::vector<Blk> m;
    for (auto& b : A.freel) {
      if (!m.empty() && m.back().off + m.back().size == b.off) m.back().size += b.size;
      else m.push_back(b);
    }
    if (!m.empty() && m.back().off + m.back().size == A.top) { A.top = m.back().off; m.pop_back(); }
    A.freel.swap(m);
  };
  std::vector<int64_t> ssa_off(L + P.steps.size(), 0);
  for (int i = 0; i < L; ++i) {
    LeafUse& U = P.leaf_use[i];
    U.off = U.phase == 0 ? U.store_off : alloc(ar[U.phase], int64_t(1) << U.sub_labels.size());
    ssa_off[i] = U.off;
  }
  // execution order: phase 0 steps, then phase 1, then phase 2 (each in tree order)
  for (int ph = 0; ph < 3; ++ph) {
    for (size_t s = 0; s < P.steps.size(); ++s) {
      Step& S = P.steps[s];
      if (S.phase != ph) continue;
      int64_t sz = int64_t(1) << S.lc.size();
      S.off_c = alloc(ar[ph], sz);
      ssa_off[L + s] = S.off_c;
      if (ph == 0) continue;  // invariant results stay
      for (int opnd : {S.a, S.b}) {
        // an operand lives in its own phase's memory; free it when consumed in that phase
        if (phase_of(opnd) == ph) release(ar[ph], ssa_off[opnd], int64_t(1) << order[opnd].size());
      }
    }
  }
  P.invariant_elems = std::max<int64_t>(ar[0].peak, 32);
  P.slice_arena_elems = align(std::max<int64_t>(ar[1].peak, 32));
  P.unit_arena_elems = align(std::max<int64_t>(ar[2].peak, 32));

  // ---- root permutation: batch index j -> element offset of the root tensor
  const LSet& root = L == 1 ? P.leaf_use[0].sub_labels : P.steps.back().lc;
  int k = (int)net.open_qubits.size();
  P.root_perm.assign(size_t(1) << k, 0);
  for (int64_t j = 0; j < (int64_t(1) << k); ++j) {
    int64_t off = 0;
    for (size_t pos = 0; pos < root.size(); ++pos) {
      int t = net.open_bit[root[pos]];
      if (t < 0) return fail(TN_EINVAL, "tn_plan: internal error, root holds a non-open label");
      if ((j >> t) & 1) off += int64_t(1) << (root.size() - 1 - pos);
    }
    P.root_perm[j] = off;
  }

  // ---- serialization + hash
  auto& b = P.bytes;
  b.clear();
  const char magic[8] = {'T', 'N', 'P', 'L', 'A', 'N', '0', '1'};
  b.insert(b.end(), magic, magic + 8);
  put32(b, net.n);
  put32(b, k);
  for (int q : net.open_qubits) put32(b, q);
  put32(b, (int)P.sliced.size());
  for (int l : P.sliced) { put32(b, net.wire[l].first); put32(b, net.wire[l].second); }
  put32(b, L);
  for (int i = 0; i < L; ++i) {
    put32(b, (int)net.leaves[i].labels.size());
    for (int l : net.leaves[i].labels) { put32(b, net.wire[l].first); put32(b, net.wire[l].second); }
  }
  put32(b, (int)P.steps.size());
  for (auto& S : P.steps) {
    put32(b, S.a);
    put32(b, S.b);
    put32(b, S.klass);
    put32(b, S.phase);
    put32(b, (int)S.lc.size());
    for (int l : S.lc) { put32(b, net.wire[l].first); put32(b, net.wire[l].second); }
  }
  P.hash = fnv1a(b);
  return TN_OK;
}

Plan::~Plan() {
  if (exec) destroy_executor(exec);
}

}  // namespace tn

using namespace tn;

extern "C" tn_status tn_plan(const tn_network* net, const tn_plan_opts* opts, tn_plan_t** out) {
  if (!net || !out) return fail(TN_EINVAL, "tn_plan: NULL argument");
  tn_plan_opts o;
  std::memset(&o, 0, sizeof o);
  o.num_sliced = -1;
  if (opts) o = *opts;
  if (o.num_sliced < -1 || o.num_sliced > 62) return fail(TN_EINVAL, "tn_plan: num_sliced %d not in [-1, 62]", o.num_sliced);
  if (o.max_log2_intermediate < 0 || o.max_log2_intermediate > 30)
    return fail(TN_EINVAL, "tn_plan: max_log2_intermediate %d not in [0, 30]", o.max_log2_intermediate);
  if (o.search_trials < 0 || o.search_trials > 100000) return fail(TN_EINVAL, "tn_plan: bad search_trials");
  if (o.cap_aware_rewrites < 0 || o.cap_aware_rewrites > 1)
    return fail(TN_EINVAL, "tn_plan: cap_aware_rewrites %d not 0 or 1", o.cap_aware_rewrites);
  return guarded("tn_plan", [&]() -> tn_status {
    std::unique_ptr<tn_plan_s> h(new tn_plan_s);
    tn_status st = make_plan(net->net, o, h->plan);
    if (st != TN_OK) return st;
    *out = h.release();
    return TN_OK;
  });
}

extern "C" tn_status tn_plan_get_info(const tn_plan_t* p, tn_plan_info* info) {
  if (!p || !info) return fail(TN_EINVAL, "tn_plan_get_info: NULL argument");
  const Plan& P = p->plan;
  std::memset(info, 0, sizeof *info);
  info->num_qubits = P.net.n;
  info->num_open = (int)P.net.open_qubits.size();
  info->num_sliced = (int)P.sliced.size();
  info->num_steps = (int)P.steps.size();
  info->num_leaves = (int)P.net.leaves.size();
  info->max_log2_intermediate = P.max_width;
  info->num_slices = num_slice_ids(P);
  info->cmac_per_slice = P.cmac_per_slice;
  info->flops_per_slice = 8.0 * P.cmac_per_slice;
  info->log2_cmac_total = std::log2(std::max(P.cmac_per_slice, 1.0)) + (double)P.sliced.size();
  info->footprint_bytes_per_unit = (P.unit_arena_elems + P.slice_arena_elems) * 8;
  info->hash = P.hash;
  for (auto& S : P.steps) {
    if (S.klass == SC_VECTOR) info->num_vector_steps++;
    else info->num_dense_steps++;
  }
  return TN_OK;
}

extern "C" tn_status tn_plan_sliced_wires(const tn_plan_t* p, int32_t* pairs, int64_t cap) {
  if (!p || (!pairs && !p->plan.sliced.empty())) return fail(TN_EINVAL, "tn_plan_sliced_wires: NULL argument");
  const Plan& P = p->plan;
  if (cap < (int64_t)P.sliced.size()) return fail(TN_EINVAL, "tn_plan_sliced_wires: capacity too small");
  for (size_t j = 0; j < P.sliced.size(); ++j) {
    pairs[2 * j] = P.net.wire[P.sliced[j]].first;
    pairs[2 * j + 1] = P.net.wire[P.sliced[j]].second;
  }
  return TN_OK;
}

extern "C" tn_status tn_plan_serialize(const tn_plan_t* p, uint8_t* buf, size_t cap, size_t* len) {
  if (!p || !len) return fail(TN_EINVAL, "tn_plan_serialize: NULL argument");
  const auto& b = p->plan.bytes;
  *len = b.size();
  if (!buf) return TN_OK;
  if (cap < b.size()) return fail(TN_EINVAL, "tn_plan_serialize: capacity %zu < %zu", cap, b.size());
  std::memcpy(buf, b.data(), b.size());
  return TN_OK;
}

extern "C" tn_status tn_plan_tree(const tn_plan_t* p, int32_t* leaf_raw, int64_t cap_raw, int32_t* tree,
                                  int64_t cap_tree) {
  if (!p || !leaf_raw || !tree) return fail(TN_EINVAL, "tn_plan_tree: NULL argument");
  const Plan& P = p->plan;
  int64_t need = 0;
  for (auto& lf : P.net.leaves) need += (int64_t)lf.raw.size() + 1;
  const int64_t need_tree = 2 * (int64_t)P.steps.size();
  if (cap_raw < need || cap_tree < need_tree)
    return fail(TN_EINVAL, "tn_plan_tree: capacity too small (need %lld raw, %lld tree)", (long long)need,
                (long long)need_tree);
  int64_t k = 0;
  for (auto& lf : P.net.leaves) {
    for (int r : lf.raw) leaf_raw[k++] = r;
    leaf_raw[k++] = -1;
  }
  // steps store operands as (a, b) after the size swap; report the tree in step order
  for (size_t s = 0; s < P.steps.size(); ++s) {
    tree[2 * s] = P.steps[s].a;
    tree[2 * s + 1] = P.steps[s].b;
  }
  return TN_OK;
}

extern "C" tn_status tn_plan_layout(const tn_plan_t* p, tn_tensor_layout* out, int64_t capacity,
                                    int64_t* arena_elems) {
  if (!p || !out || !arena_elems) return fail(TN_EINVAL, "tn_plan_layout: NULL argument");
  const Plan& P = p->plan;
  const int L = (int)P.net.leaves.size();
  const int64_t nt = L + (int64_t)P.steps.size();
  if (capacity < nt) return fail(TN_EINVAL, "tn_plan_layout: capacity %lld < %lld tensors", (long long)capacity,
                                 (long long)nt);
  return guarded("tn_plan_layout", [&]() -> tn_status {
    std::vector<int32_t> consumer(nt, -1);
    for (size_t s = 0; s < P.steps.size(); ++s) {
      consumer[P.steps[s].a] = (int32_t)s;
      consumer[P.steps[s].b] = (int32_t)s;
    }
    for (int i = 0; i < L; ++i) {
      const LeafUse& U = P.leaf_use[i];
      tn_tensor_layout t{};
      t.phase = U.phase;
      t.producer = -1;
      t.consumer = consumer[i];
      t.log2_elems = (int32_t)U.sub_labels.size();
      t.offset = U.off;
      t.store_offset = U.store_off;
      t.store_log2 = (int32_t)P.net.leaves[i].labels.size();
      t.step_class = t.log2_m = t.log2_n = t.log2_k = -1;
      out[i] = t;
    }
    for (size_t s = 0; s < P.steps.size(); ++s) {
      tn_tensor_layout t{};
      t.phase = P.steps[s].phase;
      t.producer = (int32_t)s;
      t.consumer = consumer[L + s];
      t.log2_elems = (int32_t)P.steps[s].lc.size();
      t.offset = P.steps[s].off_c;
      t.store_offset = -1;
      t.store_log2 = -1;
      t.step_class = P.steps[s].klass;
      t.log2_m = P.steps[s].nm;
      t.log2_n = P.steps[s].nn;
      t.log2_k = P.steps[s].nk;
      out[L + s] = t;
    }
    arena_elems[0] = P.leaf_store_elems;
    arena_elems[1] = P.invariant_elems;
    arena_elems[2] = P.slice_arena_elems;
    arena_elems[3] = P.unit_arena_elems;
    return TN_OK;
  });
}
