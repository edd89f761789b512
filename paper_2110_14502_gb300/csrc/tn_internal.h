// Internal data structures of the host library (circuits, networks, plans).
#pragma once

#include <complex>
#include <cstdint>
#include <exception>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "tn.h"

namespace tn {

using cd = std::complex<double>;

// Records a printf-style message for tn_last_error() and returns `code`.
tn_status fail(tn_status code, const char* fmt, ...);

// Runs an entry point's body (a callable returning tn_status) so that no C++
// exception crosses the C ABI: a failed host allocation becomes TN_ENOMEM,
// any other exception TN_EINTERNAL with its message.
template <class F>
tn_status guarded(const char* fn, F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return fail(TN_ENOMEM, "%s: out of host memory", fn);
  } catch (const std::exception& e) {
    return fail(TN_EINTERNAL, "%s: %s", fn, e.what());
  } catch (...) {
    return fail(TN_EINTERNAL, "%s: unexpected exception", fn);
  }
}

struct Gate {
  int kind = 0;
  int q0 = 0, q1 = -1;
  double theta = 0, phi = 0;
  cd m[16];  // row-major 2x2 (first 4) or 4x4
  int nq() const { return q1 < 0 ? 1 : 2; }
};

struct Circuit {
  int n = 0;
  int cols = 0;  // grid width of a generated circuit (qubit q at row q / cols, column q % cols); 0 = unknown
  std::vector<Gate> gates;
};

// Fills g.m from g.kind/theta/phi for the named kinds.
void gate_matrix(Gate& g);
uint64_t splitmix64_next(uint64_t& state);

enum LabelKind { LK_INTERNAL = 0, LK_OPEN = 1, LK_CLOSED = 2 };

struct Leaf {
  std::vector<int> labels;  // row-major order, first label slowest
  std::vector<cd> data;     // 2^labels.size()
  std::vector<int> raw;     // raw tensor ids merged into this leaf
};

struct Network {
  int n = 0;
  int cols = 0;  // grid width of the circuit, 0 = unknown
  int num_gates = 0;
  std::vector<int> open_qubits;
  std::vector<Leaf> leaves;
  std::vector<std::pair<int, int>> wire;  // label -> (q, t)
  std::vector<int> kind;                  // label -> LabelKind
  std::vector<int> closed_qubit;          // label -> qubit (LK_CLOSED) else -1
  std::vector<int> open_bit;              // label -> bit of the batch index (LK_OPEN) else -1
  int num_labels() const { return (int)wire.size(); }
};

// Kernel class of a pairwise step.
enum StepClass { SC_SIMT = 0, SC_VECTOR = 1, SC_TC = 2 };

struct Step {
  int a = -1, b = -1;           // SSA operand ids: < L leaf, else L + step index
  std::vector<int> la, lb, lc;  // operand / output labels in memory order (fixed labels removed)
  int nm = 0, nn = 0, nk = 0;   // log2 M, N, K
  int klass = SC_SIMT;
  bool variant = true;          // depends on the unit's fixed-index values
  int phase = 2;                // 0 invariant, 1 slice-only, 2 per (bitstring, slice)
  int64_t off_c = 0;            // element offset of the output in its phase's memory
};

struct LeafUse {
  bool variant = false;
  int phase = 0;                // 0 invariant (leaf store), 1 slice arena, 2 pair arena
  std::vector<int> sub_labels;  // labels after removing fixed ones
  // per full-label position: -1 kept, else source of the fixed value:
  //   src >= 0      : sliced index number j (bit j of the slice id)
  //   src <= -2     : closed output of qubit (-src - 2)
  std::vector<int> fixed_src;
  int64_t off = 0;              // variant: element offset in unit arena; invariant: offset in leaf store
  int64_t store_off = 0;        // offset of the full leaf in the leaf store
};

struct Executor;   // device-side state (executor.cu)
struct StemCache;  // device-resident stems shared by plan copies (executor.cu)

struct PlanData {
  Network net;
  tn_plan_opts opts{};
  std::vector<int> sliced;      // labels; bit j of the slice id -> sliced[j]
  std::vector<int> tree;        // 2*(L-1) SSA ids
  std::vector<Step> steps;
  std::vector<LeafUse> leaf_use;
  int64_t unit_arena_elems = 0;   // per-(bitstring, slice) arena (complex elements)
  int64_t slice_arena_elems = 0;  // per-slice arena for slice-only tensors
  int64_t invariant_elems = 0;    // invariant intermediates store
  int64_t leaf_store_elems = 0;
  std::vector<int64_t> root_perm; // batch index j -> element offset in the root tensor
  double cmac_per_slice = 0;
  double cmac_slice_only = 0;     // part of cmac_per_slice shared by every bitstring of a slice
  int max_width = 0;
  std::vector<uint8_t> bytes;     // serialized form
  uint64_t hash = 0;
};

// Slice ids a call can address: 2^S, or 2^62 when S >= 62 (ids are int64_t;
// bit j of the id fixes sliced index j, so higher sliced indices of a plan
// with S >= 62 stay at 0 -- a leading range of the 2^S slices).
inline int64_t num_slice_ids(const PlanData& P) {
  return P.sliced.size() >= 62 ? int64_t(1) << 62 : int64_t(1) << P.sliced.size();
}

// A plan plus its device state.  Copies share nothing on the device: a copy
// starts without an executor and allocates its own on first use.
struct Plan : PlanData {
  Executor* exec = nullptr;
  // When set, the plan's stem (leaf store and phase-0 outputs, which depend
  // on neither the bitstring nor the slice) comes from this cache and is
  // shared with every other plan of the same circuit that uses it.
  std::shared_ptr<StemCache> stems;
  Plan() = default;
  Plan(const Plan& o) : PlanData(o), exec(nullptr) {}
  Plan& operator=(const Plan&) = delete;
  ~Plan();
};

// network.cpp
tn_status build_network(const Circuit& c, const int32_t* open, int num_open, Network& out, int flags = 0);
// planner.cpp
tn_status make_plan(const Network& net, const tn_plan_opts& opts, Plan& plan);
// executor.cu
void destroy_executor(Executor* e);
tn_status contract_amplitudes(Plan& p, const uint64_t* bits, int64_t nb, double* out,
                              const tn_exec_opts& o, tn_report* rep);
// As above; clear_out = false adds into `out` (device I/O) instead of
// overwriting it.  flags: bit 0 = reset the list of filter-flagged units at
// the start, bit 1 = run the filter (recompute / discard) at the end; a caller
// splitting one sum over several calls resets on the first and filters on the last.
tn_status contract_amplitudes_ex(Plan& p, const uint64_t* bits, int64_t nb, double* out, const tn_exec_opts& o,
                                 tn_report* rep, bool clear_out, int flags);
// Device bytes held by the plan's executor (0 before its first use).
int64_t executor_bytes(const Plan& p);
// Stem cache of one server: entries keyed by (device, plan hash), each the
// leaf store and phase-0 outputs of a plan.  Entries no plan uses any more
// are evicted least recently used first once the cache holds more than
// cap_bytes.
std::shared_ptr<StemCache> make_stem_cache(int64_t cap_bytes);
// Whether the plan's last call found its phase-0 outputs already computed by
// another plan sharing its stem.
bool stem_reused(const Plan& p);
struct StemCacheStats { int64_t entries, bytes, hits, misses; };
StemCacheStats stem_cache_stats(StemCache& c);

}  // namespace tn

struct tn_circuit_s { tn::Circuit c; };
struct tn_network_s { tn::Network net; };
struct tn_plan_s {
  tn::Plan plan;
  tn_plan_s() = default;
  explicit tn_plan_s(const tn::Plan& p) : plan(p) {}
};
