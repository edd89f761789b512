// Tensor network of <x|U|0^n> (paper: Sec. "Existing Efforts on Simulation of
// RQCs" -- a one-qubit gate is a rank-2 tensor, a two-qubit gate a rank-4
// tensor), with closed output wires kept as fixed indices and small tensors
// absorbed into neighbours.
//
// Diagonal decomposition (option TN_NET_SPLIT_DIAGONAL; paper: Sec. "A
// PEPS-based Simulation Method with an Optimized Slicing Strategy", where
// diagonal gates make their wire indices hyperedges).  A two-qubit gate that
// is a wire swap times a diagonal -- fSim(pi/2, phi) = SWAP diag(1, -i, -i,
// e^{-i phi}) -- needs no tensor of its own: the swap renames the wires (the
// input index of qubit a continues as the wire of qubit b and vice versa)
// and the diagonal D(x_a, x_b) would make both wire indices hyperedges.  D has
// operator-Schmidt rank 2, D(x, y) = sum_c delta(x, c) D(c, y), so its two
// factors go into the tensors that produced the two wires: the producer of
// x_a gains the bond index c as a copy of x_a, the producer of x_b the factor
// D(c, x_b).  Every index keeps exactly two holders.
#include <algorithm>
#include <cstring>
#include <map>

#include "tn_internal.h"

namespace tn {

// Host FP64 pairwise contraction of small tensors.  Result labels: U's
// unshared labels, then T's unshared labels.
static Leaf contract_small(const Leaf& U, const Leaf& T) {
  Leaf R;
  std::vector<int> shared;
  for (int l : U.labels)
    if (std::find(T.labels.begin(), T.labels.end(), l) != T.labels.end()) shared.push_back(l);
  for (int l : U.labels)
    if (std::find(shared.begin(), shared.end(), l) == shared.end()) R.labels.push_back(l);
  for (int l : T.labels)
    if (std::find(shared.begin(), shared.end(), l) == shared.end()) R.labels.push_back(l);
  std::vector<int> uni = R.labels;
  uni.insert(uni.end(), shared.begin(), shared.end());
  const int nu = (int)uni.size(), nr = (int)R.labels.size();
  auto pos_in = [&](const std::vector<int>& ls, int l) {
    for (size_t i = 0; i < ls.size(); ++i)
      if (ls[i] == l) return (int)i;
    return -1;
  };
  // stride of each union label within U, T, R
  std::vector<int64_t> su(nu, 0), st(nu, 0), sr(nu, 0);
  for (int i = 0; i < nu; ++i) {
    int p;
    if ((p = pos_in(U.labels, uni[i])) >= 0) su[i] = int64_t(1) << (U.labels.size() - 1 - p);
    if ((p = pos_in(T.labels, uni[i])) >= 0) st[i] = int64_t(1) << (T.labels.size() - 1 - p);
    if ((p = pos_in(R.labels, uni[i])) >= 0) sr[i] = int64_t(1) << (R.labels.size() - 1 - p);
  }
  R.data.assign(size_t(1) << nr, cd(0, 0));
  for (int64_t x = 0; x < (int64_t(1) << nu); ++x) {
    int64_t ou = 0, ot = 0, orr = 0;
    for (int i = 0; i < nu; ++i)
      if ((x >> i) & 1) { ou += su[i]; ot += st[i]; orr += sr[i]; }
    R.data[orr] += U.data[ou] * T.data[ot];
  }
  R.raw = U.raw;
  R.raw.insert(R.raw.end(), T.raw.begin(), T.raw.end());
  return R;
}

// True when the 4x4 matrix m (basis 2 x_a + x_b) is a swap times a diagonal:
// its only non-zeros are m[00,00], m[01,10], m[10,01], m[11,11].
static bool swap_times_diagonal(const cd* m) {
  double off = 0;
  for (int r = 0; r < 4; ++r)
    for (int col = 0; col < 4; ++col) {
      const int swapped = ((col & 1) << 1) | (col >> 1);
      if (r != swapped) off += std::abs(m[r * 4 + col]);
    }
  return off < 1e-12;
}

tn_status build_network(const Circuit& c, const int32_t* open, int num_open, Network& net, int flags) {
  const int n = c.n;
  net = Network();
  net.n = n;
  net.cols = c.cols;
  net.num_gates = (int)c.gates.size();
  net.open_qubits.assign(open, open + num_open);
  std::vector<int> seg(n, 0), cur(n, -1);
  auto new_label = [&](int q, int t) {
    net.wire.push_back({q, t});
    net.kind.push_back(LK_INTERNAL);
    net.closed_qubit.push_back(-1);
    net.open_bit.push_back(-1);
    return (int)net.wire.size() - 1;
  };
  std::vector<Leaf> leaves;
  std::vector<int> producer;  // label -> leaf that holds it as an output index
  auto set_producer = [&](int l, int leaf) {
    if ((int)producer.size() <= l) producer.resize(l + 1, -1);
    producer[l] = leaf;
  };
  for (int q = 0; q < n; ++q) {
    cur[q] = new_label(q, 0);
    set_producer(cur[q], (int)leaves.size());
    Leaf L;
    L.labels = {cur[q]};
    L.data = {cd(1, 0), cd(0, 0)};
    L.raw = {net.num_gates + q};
    leaves.push_back(L);
  }
  for (int i = 0; i < net.num_gates; ++i) {
    const Gate& g = c.gates[i];
    Leaf L;
    L.raw = {i};
    if (g.nq() == 1) {
      int lin = cur[g.q0];
      int lout = new_label(g.q0, ++seg[g.q0]);
      cur[g.q0] = lout;
      L.labels = {lout, lin};
      L.data.assign(g.m, g.m + 4);
      set_producer(lout, (int)leaves.size());
    } else if ((flags & TN_NET_SPLIT_DIAGONAL) && swap_times_diagonal(g.m)) {
      const int ain = cur[g.q0], bin = cur[g.q1];
      // D(x_a, x_b): the gate maps |x_a x_b> to D(x_a, x_b) |x_b x_a>
      auto D = [&](int x, int y) { return g.m[(2 * y + x) * 4 + 2 * x + y]; };
      const int pa = producer[ain], pb = producer[bin];
      auto pos = [](const Leaf& F, int l) {
        int p = 0;
        while (F.labels[p] != l) ++p;
        return p;
      };
      // raw ids of the two factors (after the gates and the inputs)
      const int raw_a = net.num_gates + n + 2 * i, raw_b = raw_a + 1;
      if (pa == pb) {  // one tensor produced both wires: D goes in whole
        Leaf& F = leaves[pa];
        const int r = (int)F.labels.size(), ia = pos(F, ain), ib = pos(F, bin);
        for (size_t e = 0; e < F.data.size(); ++e) F.data[e] *= D((e >> (r - 1 - ia)) & 1, (e >> (r - 1 - ib)) & 1);
        F.raw.push_back(raw_a);
        F.raw.push_back(raw_b);
      } else {
        const int bond = new_label(-1 - i, 0);
        for (int side = 0; side < 2; ++side) {
          Leaf& F = leaves[side ? pb : pa];
          const int r = (int)F.labels.size(), ip = pos(F, side ? bin : ain);
          std::vector<cd> nd(F.data.size() * 2);
          for (size_t e = 0; e < F.data.size(); ++e) {
            const int w = (int)((e >> (r - 1 - ip)) & 1);
            for (int cc = 0; cc < 2; ++cc) nd[2 * e + cc] = F.data[e] * (side ? D(cc, w) : cd(w == cc ? 1.0 : 0.0, 0.0));
          }
          F.data.swap(nd);
          F.labels.push_back(bond);
          F.raw.push_back(side ? raw_b : raw_a);
        }
      }
      cur[g.q0] = bin;
      cur[g.q1] = ain;
      continue;
    } else {
      int ain = cur[g.q0], bin = cur[g.q1];
      int aout = new_label(g.q0, ++seg[g.q0]);
      int bout = new_label(g.q1, ++seg[g.q1]);
      cur[g.q0] = aout;
      cur[g.q1] = bout;
      L.labels = {aout, bout, ain, bin};  // T[xa',xb',xa,xb] = m[(2xa'+xb')*4 + 2xa+xb]
      L.data.assign(g.m, g.m + 16);
      set_producer(aout, (int)leaves.size());
      set_producer(bout, (int)leaves.size());
    }
    leaves.push_back(L);
  }
  for (int q = 0; q < n; ++q) {
    int t = -1;
    for (int k = 0; k < num_open; ++k)
      if (open[k] == q) t = k;
    if (t >= 0) {
      net.kind[cur[q]] = LK_OPEN;
      net.open_bit[cur[q]] = t;
    } else {
      net.kind[cur[q]] = LK_CLOSED;
      net.closed_qubit[cur[q]] = q;
    }
  }
  // Absorb tensors of topological rank <= 2 (closed outputs do not count)
  // into the neighbour sharing the most labels (ties: lowest index).
  std::vector<char> alive(leaves.size(), 1);
  std::map<int, std::vector<int>> holders;
  for (size_t i = 0; i < leaves.size(); ++i)
    for (int l : leaves[i].labels) holders[l].push_back((int)i);
  auto topo_rank = [&](const Leaf& L) {
    int r = 0;
    for (int l : L.labels) r += net.kind[l] != LK_CLOSED;
    return r;
  };
  bool changed = true;
  while (changed) {
    changed = false;
    for (size_t i = 0; i < leaves.size(); ++i) {
      if (!alive[i] || topo_rank(leaves[i]) > 2) continue;
      int best = -1, best_shared = 0;
      for (int l : leaves[i].labels) {
        for (int j : holders[l]) {
          if (j == (int)i || !alive[j]) continue;
          int sh = 0;
          for (int x : leaves[i].labels)
            for (int y : leaves[j].labels) sh += (x == y);
          if (sh > best_shared || (sh == best_shared && j < best)) { best = j; best_shared = sh; }
        }
      }
      if (best < 0) continue;
      Leaf R = contract_small(leaves[best], leaves[i]);
      for (int l : leaves[i].labels) {
        auto& h = holders[l];
        h.erase(std::remove(h.begin(), h.end(), (int)i), h.end());
      }
      for (int l : leaves[best].labels) {
        auto& h = holders[l];
        h.erase(std::remove(h.begin(), h.end(), best), h.end());
      }
      alive[i] = 0;
      leaves[best] = std::move(R);
      for (int l : leaves[best].labels) holders[l].push_back(best);
      changed = true;
    }
  }
  for (size_t i = 0; i < leaves.size(); ++i)
    if (alive[i]) net.leaves.push_back(std::move(leaves[i]));
  return TN_OK;
}

}  // namespace tn

using namespace tn;

extern "C" tn_status tn_build_network_ex(const tn_circuit* c, const int32_t* open, int32_t num_open, int32_t flags,
                                         tn_network** out) {
  if (!c || !out) return fail(TN_EINVAL, "tn_build_network: NULL argument");
  if (flags & ~TN_NET_SPLIT_DIAGONAL) return fail(TN_EINVAL, "tn_build_network: unknown flags 0x%x", flags);
  if (num_open < 0 || num_open > 30 || (num_open > 0 && !open))
    return fail(TN_EINVAL, "tn_build_network: num_open %d not in [0, 30] or open_qubits NULL", num_open);
  for (int i = 0; i < num_open; ++i) {
    if (open[i] < 0 || open[i] >= c->c.n)
      return fail(TN_EINVAL, "tn_build_network: open qubit %d out of range", open[i]);
    for (int j = 0; j < i; ++j)
      if (open[j] == open[i]) return fail(TN_EINVAL, "tn_build_network: open qubit %d repeated", open[i]);
  }
  return guarded("tn_build_network", [&]() -> tn_status {
    std::unique_ptr<tn_network_s> h(new tn_network_s);
    tn_status st = build_network(c->c, open, num_open, h->net, flags);
    if (st != TN_OK) return st;
    *out = h.release();
    return TN_OK;
  });
}

extern "C" tn_status tn_build_network(const tn_circuit* c, const int32_t* open, int32_t num_open,
                                      tn_network** out) {
  return tn_build_network_ex(c, open, num_open, 0, out);
}

extern "C" tn_status tn_network_get_info(const tn_network* net, tn_network_info* info) {
  if (!net || !info) return fail(TN_EINVAL, "tn_network_get_info: NULL argument");
  const Network& N = net->net;
  info->num_qubits = N.n;
  info->num_open = (int)N.open_qubits.size();
  info->num_leaves = (int)N.leaves.size();
  info->num_labels = N.num_labels();
  int mr = 0;
  for (auto& L : N.leaves) mr = std::max(mr, (int)L.labels.size());
  info->max_leaf_rank = mr;
  int nc = 0;
  for (int k : N.kind) nc += k == LK_CLOSED;
  info->num_closed = nc;
  return TN_OK;
}

extern "C" tn_status tn_network_label_wires(const tn_network* net, int32_t* pairs, int64_t cap) {
  if (!net || !pairs) return fail(TN_EINVAL, "tn_network_label_wires: NULL argument");
  const Network& N = net->net;
  if (cap < N.num_labels()) return fail(TN_EINVAL, "tn_network_label_wires: capacity too small");
  for (int l = 0; l < N.num_labels(); ++l) {
    pairs[2 * l] = N.wire[l].first;
    pairs[2 * l + 1] = N.wire[l].second;
  }
  return TN_OK;
}

extern "C" void tn_free_network(tn_network* net) { delete net; }
