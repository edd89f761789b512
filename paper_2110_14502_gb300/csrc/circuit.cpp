// Circuits: gate matrices and the seeded random-circuit protocol
// (paper: Sec. "General Background of RQC"; the gate set is the benchmark's,
// with fSim named in Sec. "Searching for Better Contraction Paths").
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "tn_internal.h"

namespace tn {

static thread_local std::string g_last_error;

tn_status fail(tn_status code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

const char* last_error() { return g_last_error.c_str(); }

// SplitMix64 (Steele, Lea, Flood 2014).
uint64_t splitmix64_next(uint64_t& s) {
  s += 0x9E3779B97F4A7C15ull;
  uint64_t z = s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint32_t uniform_below(uint64_t& s, uint32_t k) {
  return (uint32_t)(((splitmix64_next(s) >> 32) * (uint64_t)k) >> 32);
}

void gate_matrix(Gate& g) {
  const double r = 1.0 / std::sqrt(2.0);
  const cd I(0, 1);
  for (auto& x : g.m) x = 0;
  switch (g.kind) {
    case TN_GATE_SQRTX:
      g.m[0] = r; g.m[1] = -I * r; g.m[2] = -I * r; g.m[3] = r; break;
    case TN_GATE_SQRTY:
      g.m[0] = r; g.m[1] = -r; g.m[2] = r; g.m[3] = r; break;
    case TN_GATE_SQRTW:
      g.m[0] = r; g.m[1] = -std::exp(I * (M_PI / 4)) * r;
      g.m[2] = std::exp(-I * (M_PI / 4)) * r; g.m[3] = r; break;
    case TN_GATE_FSIM: {
      double c = std::cos(g.theta), s = std::sin(g.theta);
      g.m[0] = 1; g.m[5] = c; g.m[6] = -I * s; g.m[9] = -I * s; g.m[10] = c;
      g.m[15] = std::exp(-I * g.phi);
      break;
    }
    default: break;  // MAT1 / MAT2 carry their own matrix
  }
}

// Coupler pattern p (0:A 1:B 2:C 3:D) of a rows x cols grid, pairs (a < b).
static void pattern_pairs(int rows, int cols, int p, std::vector<std::pair<int, int>>& out) {
  out.clear();
  if (p < 2) {
    for (int r = 0; r < rows; ++r)
      for (int c = p; c + 1 < cols; c += 2) out.push_back({r * cols + c, r * cols + c + 1});
  } else {
    for (int r = p - 2; r + 1 < rows; r += 2)
      for (int c = 0; c < cols; ++c) out.push_back({r * cols + c, (r + 1) * cols + c});
  }
}

}  // namespace tn

using namespace tn;

extern "C" const char* tn_last_error(void) { return tn::last_error(); }
extern "C" const char* tn_version(void) { return "gb300-rqc-tn 0.1"; }

extern "C" tn_status tn_random_circuit(int32_t rows, int32_t cols, int32_t depth, uint64_t seed,
                                       tn_circuit** out) {
  if (!out) return fail(TN_EINVAL, "tn_random_circuit: out is NULL");
  if (rows < 1 || cols < 1 || rows > 64 || cols > 64 || rows * cols > 64 || depth < 0 || depth > 4096)
    return fail(TN_EINVAL, "tn_random_circuit: bad grid %dx%d depth %d", rows, cols, depth);
  return guarded("tn_random_circuit", [&]() -> tn_status {
  std::unique_ptr<tn_circuit_s> h(new tn_circuit_s);
  Circuit& C = h->c;
  C.n = rows * cols;
  C.cols = cols;
  uint64_t s = seed;
  std::vector<int> prev(C.n, -1);
  auto one_qubit_layer = [&]() {
    for (int q = 0; q < C.n; ++q) {
      int kind;
      if (prev[q] < 0) {
        kind = (int)uniform_below(s, 3);
      } else {
        int opts[2], k = 0;
        for (int x = 0; x < 3; ++x)
          if (x != prev[q]) opts[k++] = x;
        kind = opts[uniform_below(s, 2)];
      }
      prev[q] = kind;
      Gate g;
      g.kind = kind; g.q0 = q; g.q1 = -1;
      gate_matrix(g);
      C.gates.push_back(g);
    }
  };
  one_qubit_layer();
  std::vector<std::pair<int, int>> pairs;
  for (int c = 0; c < depth; ++c) {
    pattern_pairs(rows, cols, c % 4, pairs);
    for (auto& pr : pairs) {
      Gate g;
      g.kind = TN_GATE_FSIM; g.q0 = pr.first; g.q1 = pr.second;
      g.theta = M_PI / 2; g.phi = M_PI / 6;
      gate_matrix(g);
      C.gates.push_back(g);
    }
    one_qubit_layer();
  }
  *out = h.release();
  return TN_OK;
  });
}

extern "C" tn_status tn_circuit_from_gates(int32_t n, int64_t num_gates, const tn_gate* gates,
                                           tn_circuit** out) {
  if (!out) return fail(TN_EINVAL, "tn_circuit_from_gates: out is NULL");
  if (n < 1 || n > 64) return fail(TN_EINVAL, "tn_circuit_from_gates: num_qubits %d not in [1, 64]", n);
  if (num_gates < 0 || (num_gates > 0 && !gates))
    return fail(TN_EINVAL, "tn_circuit_from_gates: bad gate array");
  return guarded("tn_circuit_from_gates", [&]() -> tn_status {
  std::unique_ptr<tn_circuit_s> h(new tn_circuit_s);
  h->c.n = n;
  for (int64_t i = 0; i < num_gates; ++i) {
    const tn_gate& t = gates[i];
    Gate g;
    g.kind = t.kind; g.q0 = t.q0; g.q1 = t.q1; g.theta = t.theta; g.phi = t.phi;
    bool two = (t.kind == TN_GATE_FSIM || t.kind == TN_GATE_MAT2);
    bool known = t.kind >= TN_GATE_SQRTX && t.kind <= TN_GATE_MAT2;
    if (!known || t.q0 < 0 || t.q0 >= n || (two && (t.q1 < 0 || t.q1 >= n || t.q1 == t.q0)))
      return fail(TN_EINVAL, "tn_circuit_from_gates: gate %lld has bad kind/qubits", (long long)i);
    if (!two) g.q1 = -1;
    if (t.kind == TN_GATE_MAT1 || t.kind == TN_GATE_MAT2) {
      int d = two ? 4 : 2;
      for (int e = 0; e < d * d; ++e) g.m[e] = cd(t.mat[2 * e], t.mat[2 * e + 1]);
    } else {
      gate_matrix(g);
    }
    h->c.gates.push_back(g);
  }
  *out = h.release();
  return TN_OK;
  });
}

extern "C" tn_status tn_circuit_info(const tn_circuit* c, int32_t* n, int64_t* ng) {
  if (!c || !n || !ng) return fail(TN_EINVAL, "tn_circuit_info: NULL argument");
  *n = c->c.n;
  *ng = (int64_t)c->c.gates.size();
  return TN_OK;
}

extern "C" tn_status tn_circuit_gates(const tn_circuit* c, tn_gate* out, int64_t cap) {
  if (!c || !out) return fail(TN_EINVAL, "tn_circuit_gates: NULL argument");
  if (cap < (int64_t)c->c.gates.size()) return fail(TN_EINVAL, "tn_circuit_gates: capacity too small");
  for (size_t i = 0; i < c->c.gates.size(); ++i) {
    const Gate& g = c->c.gates[i];
    tn_gate t;
    std::memset(&t, 0, sizeof t);
    t.kind = g.kind; t.q0 = g.q0; t.q1 = g.q1; t.theta = g.theta; t.phi = g.phi;
    int d = g.nq() == 2 ? 4 : 2;
    for (int e = 0; e < d * d; ++e) { t.mat[2 * e] = g.m[e].real(); t.mat[2 * e + 1] = g.m[e].imag(); }
    out[i] = t;
  }
  return TN_OK;
}

extern "C" void tn_free_circuit(tn_circuit* c) { delete c; }
