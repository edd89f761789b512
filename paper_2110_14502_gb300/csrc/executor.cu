// Executor: runs a plan's step chain over groups of (bitstring, slice) units
// and sums the unit results in FP64 (paper: Sec. "A Customized Parallelization
// Scheme" -- slices are independent sub-tasks, here the units of one GPU's
// work instead of MPI processes -- and Sec. "Scaling", global reduction).
//
// Steps run in three phases.  Phase 0 (no fixed index below the step) runs
// once per plan.  Phase 1 (depends on sliced indices only) runs once per
// slice and its results are shared by every bitstring of the call.  Phase 2
// (depends on the bitstring's closed output bits) runs once per (bitstring,
// slice) unit.  A launch covers a whole group of units (grid dimension), with
// shared operands addressed through zero unit strides.
//
// Device memory of a plan (allocated on first use, kept until tn_free_plan):
//   leaf store   -- every leaf tensor in complex64, full (fixed indices included)
//   invariant    -- outputs of phase-0 steps
//                   (these two come from the server's stem cache when the plan
//                   is a serving copy: shared by the plans of one circuit)
//   slice arena  -- Gs slices x per-slice arena (phase-1 leaves and outputs)
//   pair arena   -- Gs x Gb units x per-unit arena (phase-2 leaves and outputs)
//   accumulator  -- nb x 2^k complex128 (host I/O; device I/O sums into `out`)
//   scratch      -- 16-bit operand planes of the tensor-core steps
//   scale pool   -- exponents, maxima and flags of the scaled precisions
// The arenas, scratch and pool only grow; growing one drops the recorded
// CUDA graphs, which hold their addresses.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kernels.h"
#include "tn_internal.h"

namespace tn {

constexpr int kFlaggedCap = 1 << 16;  // listed flagged units per call
// Default of the plane handover per precision (c64, split bf16, split fp16,
// scaled fp16, scaled bf16).  A handed-over 16-bit tensor is scaled by the
// bound 2 K maxA maxB predicted before its values exist, so its stored
// maximum may sit a few binades below the target range; in split fp16 the lo
// plane still carries the bits the hi plane drops, and only components far
// below the maximum lose precision to fp16's subnormal range.
constexpr bool kHandoverDefault[5] = {false, true, true, true, true};

// A plan's stem: the leaf store and the phase-0 outputs.  Neither depends on
// the bitstring, the slice or the precision (phase 0 always runs in
// complex64), so every plan of one circuit can read the same copy.  A stem
// is identified by the plan's hash and by a hash of its leaf tensors' values:
// circuits of the same grid and depth drawn with different seeds have the
// same structure, hence the same plan, but different gate matrices.  The
// first plan that needs the phase-0 outputs computes them on its stream and
// records `ready`; later plans make their streams wait for that event.
struct Stem {
  int device = -1;
  uint64_t hash = 0, data_hash = 0;
  float2* store = nullptr;
  float2* inv = nullptr;
  int64_t bytes = 0;
  std::mutex mu;
  bool inv_ready = false;
  cudaEvent_t ready = nullptr;
  ~Stem() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (device >= 0) cudaSetDevice(device);
    cudaFree(store);
    cudaFree(inv);
    if (ready) cudaEventDestroy(ready);
    if (cur >= 0) cudaSetDevice(cur);
  }
};

struct StemCache {
  std::mutex mu;
  int64_t cap = 0, bytes = 0, hits = 0, misses = 0;
  uint64_t tick = 0;
  struct Entry { std::shared_ptr<Stem> stem; uint64_t last = 0; };
  std::map<std::tuple<int, uint64_t, uint64_t>, Entry> m;  // (device, plan hash, leaf data hash)
};

std::shared_ptr<StemCache> make_stem_cache(int64_t cap_bytes) {
  auto c = std::make_shared<StemCache>();
  c->cap = std::max<int64_t>(0, cap_bytes);
  return c;
}

StemCacheStats stem_cache_stats(StemCache& c) {
  std::lock_guard<std::mutex> g(c.mu);
  return {(int64_t)c.m.size(), c.bytes, c.hits, c.misses};
}

struct Executor {
  int device = -1;
  float2* store = nullptr;
  float2* inv = nullptr;
  bool inv_ready = false;
  std::shared_ptr<Stem> stem;  // when set, store and inv belong to it
  bool stem_reused = false;
  float2* sarena = nullptr;  // slice arena
  float2* parena = nullptr;  // pair arena
  int64_t sarena_cap = 0, parena_cap = 0;  // capacities in elements
  LeafGather* gather = nullptr;  // phase-1 descriptors then phase-2 descriptors
  int ngather1 = 0, ngather2 = 0;
  int64_t* perm = nullptr;
  uint64_t* bits = nullptr;
  int64_t bits_cap = 0;
  double2* acc = nullptr;
  int64_t acc_cap = 0;
  int* err = nullptr;          // device error word of bounded waits
  uint16_t* scratch = nullptr; // split operand planes of the tensor-core steps
  int64_t scratch_cap = 0;     // in 16-bit elements
  // scaled precisions: per step and launch unit, exponent and stored maximum
  // of plane outputs; per split role the same plus the max reduction; flags
  uint8_t* spool = nullptr;
  int64_t spool_cap = 0;       // bytes
  int64_t* flagged = nullptr;  // (b << 32 | s) of units kept out of the sum
  unsigned long long* nflagged = nullptr;
  GroupInfo* gslot = nullptr;  // [2]: group of the slice-only launches, group of the per-unit launches
  // replayable launch sequences, keyed by (phase, precision, plane handover,
  // Gs, Gb); dropped whenever a buffer they reference is reallocated
  struct Graph { int phase, precision, handover, gs, gb; cudaGraphExec_t exec; int64_t kernels; };
  std::vector<Graph> graphs;
  // autotuner choices per (precision, step): tensor-core tile width, raster group
  struct Tune { int precision, step, tile_n, group_m, persistent; };
  std::vector<Tune> tuned;
  bool tune_loaded = false;
  std::vector<GemmDesc> desc;  // per step, unit strides filled at launch
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> pev;  // profiling event pool
};

void destroy_executor(Executor* e) {
  if (!e) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (e->device >= 0) cudaSetDevice(e->device);
  if (!e->stem) {
    cudaFree(e->store);
    cudaFree(e->inv);
  }
  e->stem.reset();
  cudaFree(e->sarena);
  cudaFree(e->parena);
  cudaFree(e->gather);
  cudaFree(e->perm);
  cudaFree(e->bits);
  cudaFree(e->acc);
  cudaFree(e->err);
  cudaFree(e->scratch);
  cudaFree(e->spool);
  cudaFree(e->flagged);
  cudaFree(e->nflagged);
  cudaFree(e->gslot);
  for (auto& g : e->graphs) cudaGraphExecDestroy(g.exec);
  if (e->ev0) cudaEventDestroy(e->ev0);
  if (e->ev1) cudaEventDestroy(e->ev1);
  for (auto ev : e->pev) cudaEventDestroy(ev);
  if (cur >= 0) cudaSetDevice(cur);
  delete e;
}

// Host-side fault injection for the tests: with TN_FAULT_ALLOC=k set, the
// k-th device allocation of the executor made since the variable took its
// current value fails as if the device were out of memory.  Every call that
// allocates checks the variable, so a test can set and clear it between calls.
cudaError_t dev_alloc(void** p, size_t bytes) {
  static std::mutex mu;
  static std::string last;
  static long count = 0;
  const char* v = getenv("TN_FAULT_ALLOC");
  {
    std::lock_guard<std::mutex> g(mu);
    if (!v) {
      last.clear();
    } else {
      if (last != v) {
        last = v;
        count = 0;
      }
      if (++count == atol(v)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
    }
  }
  return cudaMalloc(p, bytes);
}
template <typename T>
cudaError_t dev_alloc(T** p, size_t bytes) {
  void* q = nullptr;
  const cudaError_t e = dev_alloc(&q, bytes);
  *p = static_cast<T*>(q);
  return e;
}

#define CK(call)                                                                                       \
  do {                                                                                                 \
    cudaError_t _e = (call);                                                                           \
    if (_e != cudaSuccess)                                                                             \
      return fail(TN_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__, __LINE__);    \
  } while (0)

// Per-bit strides of the GEMM view of one step (see GemmDesc): bits of each
// group are numbered from the operand's fastest index upward.
void make_gemm_desc(const std::vector<int>& la, const std::vector<int>& lb, const std::vector<int>& lc,
                    GemmDesc& d, bool m_by_output) {
  std::memset(&d, 0, sizeof d);
  auto stride_in = [](const std::vector<int>& ls, int l) -> int32_t {
    for (size_t p = 0; p < ls.size(); ++p)
      if (ls[p] == l) return int32_t(1) << (ls.size() - 1 - p);
    return -1;
  };
  if (m_by_output) {
    // M bits from the output's fastest M index upward (stores coalesce across
    // threads; the bandwidth kernel reads each row's K values as one run)
    for (int p = (int)lc.size() - 1; p >= 0; --p) {
      int l = lc[p];
      if (stride_in(la, l) < 0) continue;
      d.am[d.nm] = stride_in(la, l);
      d.cm[d.nm] = stride_in(lc, l);
      ++d.nm;
    }
    for (int p = (int)la.size() - 1; p >= 0; --p) {
      int l = la[p];
      int32_t sb = stride_in(lb, l);
      if (sb >= 0) { d.ak[d.nk] = stride_in(la, l); d.bk[d.nk] = sb; ++d.nk; }
    }
  } else {
    for (int p = (int)la.size() - 1; p >= 0; --p) {
      int l = la[p];
      int32_t sb = stride_in(lb, l);
      if (sb < 0) { d.am[d.nm] = stride_in(la, l); d.cm[d.nm] = stride_in(lc, l); ++d.nm; }
      else { d.ak[d.nk] = stride_in(la, l); d.bk[d.nk] = sb; ++d.nk; }
    }
  }
  for (int p = (int)lb.size() - 1; p >= 0; --p) {
    int l = lb[p];
    if (stride_in(la, l) < 0) { d.bn[d.nn] = stride_in(lb, l); d.cn[d.nn] = stride_in(lc, l); ++d.nn; }
  }
  d.units = d.units_lo = 1;
}

// Leaf store of a plan: every leaf in complex64 at its store offset.
static tn_status upload_leaves(const Plan& P, float2** store) {
  const Network& N = P.net;
  std::vector<float2> h_store(std::max<int64_t>(P.leaf_store_elems, 1));
  for (size_t i = 0; i < N.leaves.size(); ++i) {
    const Leaf& lf = N.leaves[i];
    for (size_t e = 0; e < lf.data.size(); ++e)
      h_store[P.leaf_use[i].store_off + e] = make_float2((float)lf.data[e].real(), (float)lf.data[e].imag());
  }
  CK(dev_alloc(store, h_store.size() * sizeof(float2)));
  CK(cudaMemcpy(*store, h_store.data(), h_store.size() * sizeof(float2), cudaMemcpyHostToDevice));
  return TN_OK;
}

// The plan's stem from its cache (created on a miss), evicting unused
// entries beyond the cache's capacity.
static tn_status acquire_stem(const Plan& P, int device, std::shared_ptr<Stem>& out) {
  StemCache& C = *P.stems;
  std::lock_guard<std::mutex> g(C.mu);
  // FNV-1a 64 over the bytes of every leaf tensor's values, in leaf order
  uint64_t dh = 0xcbf29ce484222325ull;
  for (const Leaf& lf : P.net.leaves) {
    const unsigned char* b = reinterpret_cast<const unsigned char*>(lf.data.data());
    for (size_t i = 0; i < lf.data.size() * sizeof(cd); ++i) {
      dh ^= b[i];
      dh *= 0x100000001b3ull;
    }
  }
  const auto key = std::make_tuple(device, P.hash, dh);
  auto it = C.m.find(key);
  if (it != C.m.end()) {
    it->second.last = ++C.tick;
    ++C.hits;
    out = it->second.stem;
    return TN_OK;
  }
  auto st = std::make_shared<Stem>();
  st->device = device;
  st->hash = P.hash;
  st->data_hash = dh;
  // resident stems that no plan holds are only a cache: when the device has
  // no room for a new stem they all go, and the allocation is tried once more
  auto evict_unused = [&] {
    for (auto j = C.m.begin(); j != C.m.end();) {
      if (j->second.stem.use_count() == 1) {
        C.bytes -= j->second.stem->bytes;
        j = C.m.erase(j);
      } else {
        ++j;
      }
    }
  };
  tn_status r = upload_leaves(P, &st->store);
  if (r != TN_OK) {
    cudaGetLastError();
    cudaFree(st->store);
    st->store = nullptr;
    evict_unused();
    r = upload_leaves(P, &st->store);
  }
  if (r != TN_OK) return r;
  const size_t inv_bytes = std::max<int64_t>(P.invariant_elems, 1) * sizeof(float2);
  if (dev_alloc(&st->inv, inv_bytes) != cudaSuccess) {
    cudaGetLastError();
    evict_unused();
    CK(dev_alloc(&st->inv, inv_bytes));
  }
  CK(cudaEventCreateWithFlags(&st->ready, cudaEventDisableTiming));
  st->bytes = 8 * (std::max<int64_t>(P.leaf_store_elems, 1) + std::max<int64_t>(P.invariant_elems, 1));
  ++C.misses;
  C.bytes += st->bytes;
  C.m[key] = StemCache::Entry{st, ++C.tick};
  // least recently used entries that no plan holds go first
  while (C.bytes > C.cap) {
    auto victim = C.m.end();
    for (auto j = C.m.begin(); j != C.m.end(); ++j)
      if (j->second.stem.use_count() == 1 && (victim == C.m.end() || j->second.last < victim->second.last))
        victim = j;
    if (victim == C.m.end()) break;
    C.bytes -= victim->second.stem->bytes;
    C.m.erase(victim);
  }
  out = st;
  return TN_OK;
}

bool stem_reused(const Plan& P) { return P.exec && P.exec->stem_reused; }

static tn_status setup(Plan& P, Executor& E) {
  CK(cudaGetDevice(&E.device));
  const Network& N = P.net;
  const int L = (int)N.leaves.size();
  if (P.stems) {
    tn_status r = acquire_stem(P, E.device, E.stem);
    if (r != TN_OK) return r;
    E.store = E.stem->store;
    E.inv = E.stem->inv;
  } else {
    tn_status r = upload_leaves(P, &E.store);
    if (r != TN_OK) return r;
    CK(dev_alloc(&E.inv, std::max<int64_t>(P.invariant_elems, 1) * sizeof(float2)));
  }
  std::vector<LeafGather> g1, g2;
  for (int i = 0; i < L; ++i) {
    const LeafUse& U = P.leaf_use[i];
    if (U.phase == 0) continue;
    const Leaf& lf = N.leaves[i];
    const int r = (int)lf.labels.size();
    if (r > kMaxLeafRank) return fail(TN_EINVAL, "leaf rank %d > %d", r, kMaxLeafRank);
    LeafGather d;
    std::memset(&d, 0, sizeof d);
    d.store_off = U.store_off;
    d.dst_off = U.off;
    for (int p = 0; p < r; ++p) {
      int32_t st = int32_t(1) << (r - 1 - p);
      if (U.fixed_src[p] == -1) d.kept_stride[d.nkept++] = st;
      else { d.fixed_src[d.nfixed] = U.fixed_src[p]; d.fixed_stride[d.nfixed] = st; ++d.nfixed; }
    }
    (U.phase == 1 ? g1 : g2).push_back(d);
  }
  E.ngather1 = (int)g1.size();
  E.ngather2 = (int)g2.size();
  g1.insert(g1.end(), g2.begin(), g2.end());
  if (!g1.empty()) {
    CK(dev_alloc(&E.gather, g1.size() * sizeof(LeafGather)));
    CK(cudaMemcpy(E.gather, g1.data(), g1.size() * sizeof(LeafGather), cudaMemcpyHostToDevice));
  }
  CK(dev_alloc(&E.perm, P.root_perm.size() * sizeof(int64_t)));
  CK(cudaMemcpy(E.perm, P.root_perm.data(), P.root_perm.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  E.desc.resize(P.steps.size());
  for (size_t s = 0; s < P.steps.size(); ++s) {
    // a GEMM-class step too narrow for the tensor cores whose shape the
    // streaming kernels take (K <= 4, N <= 256) runs as one of them
    make_gemm_desc(P.steps[s].la, P.steps[s].lb, P.steps[s].lc, E.desc[s], P.steps[s].klass == SC_VECTOR);
    if (P.steps[s].klass != SC_VECTOR && (!tc_shape_ok(E.desc[s]) || stream_preferred(E.desc[s])) &&
        vector_shape_ok(E.desc[s]))
      make_gemm_desc(P.steps[s].la, P.steps[s].lb, P.steps[s].lc, E.desc[s], true);
  }
  CK(cudaEventCreate(&E.ev0));
  CK(cudaEventCreate(&E.ev1));
  CK(dev_alloc(&E.err, sizeof(int)));
  CK(cudaMemset(E.err, 0, sizeof(int)));
  CK(dev_alloc(&E.flagged, kFlaggedCap * sizeof(int64_t)));
  CK(dev_alloc(&E.gslot, 2 * sizeof(GroupInfo)));
  CK(dev_alloc(&E.nflagged, sizeof(unsigned long long)));
  return TN_OK;
}

namespace {

// Geometry of the current launch group.
struct Geo {
  int gs = 1;       // slices in the group
  int gb = 1;       // bitstrings in the group (phase 2)
};

struct Ctx {
  const Plan& P;
  Executor& E;
  cudaStream_t st;
  bool profile;
  int64_t launches = 0;
  struct Rec { int klass; double flops, bytes; size_t ev; int step, nm, nn, nk; int64_t units; long long cfast; int planes, n16, ulo, uhi; };
  std::vector<Rec> recs;
  size_t nev = 0;
  int precision = TN_PREC_C64;
  bool tc = false;               // tensor-core precision
  int np = 4;                    // planes per operand: 4 split, 2 single
  bool bf16 = true;
  bool scaled = false;           // per-unit power-of-two exponents and the filter
  int64_t U = 1;                 // launch units the scale pool is laid out for
  int* ec_all = nullptr;         // [step][U]
  unsigned* mc_all = nullptr;    // [step][U]
  int* es[2] = {nullptr, nullptr};
  float* ms[2] = {nullptr, nullptr};
  unsigned* mb[2] = {nullptr, nullptr};
  int* flag1 = nullptr;          // [Gs] slice-only units
  int* flag2 = nullptr;          // [U] (bitstring, slice) units
  std::vector<char> planes_out;  // per step: output written as 16-bit planes for a tensor-core consumer
  std::vector<char> max_out;     // per step: a streaming step records its output's maxima for a scaled split
  const int8_t* step_prec = nullptr;  // per-step precision override (TN_PREC_*, -1 = the call's)
  int call_precision = TN_PREC_C64;
  bool tuning = false;           // time the tile choices of each tensor-core step
  bool sizing = false;           // only compute scratch needs (no launches)
  int64_t scratch_need = 0;
  Ctx(const Plan& p, Executor& e, cudaStream_t s, bool prof) : P(p), E(e), st(s), profile(prof) {}

  tn_status event(size_t& idx) {
    if (nev == E.pev.size()) {
      cudaEvent_t ev;
      CK(cudaEventCreate(&ev));
      E.pev.push_back(ev);
    }
    idx = nev++;
    CK(cudaEventRecord(E.pev[idx], st));
    return TN_OK;
  }
};

// Base pointer and (lo, hi) unit strides of SSA operand x inside a launch of `phase`.
void operand(const Plan& P, const Executor& E, int x, int phase, const Geo& g, const float2*& ptr, int64_t& lo,
             int64_t& hi) {
  const int L = (int)P.net.leaves.size();
  int ph;
  int64_t off;
  if (x < L) { ph = P.leaf_use[x].phase; off = P.leaf_use[x].off; }
  else { ph = P.steps[x - L].phase; off = P.steps[x - L].off_c; }
  if (ph == 0) {
    ptr = (x < L ? E.store : E.inv) + off;
    lo = hi = 0;
  } else if (ph == 1) {
    ptr = E.sarena + off;
    lo = P.slice_arena_elems;  // slice index is the low part of the unit in both phases
    hi = 0;
  } else {
    ptr = E.parena + off;
    lo = P.unit_arena_elems;
    hi = (int64_t)g.gs * P.unit_arena_elems;
  }
  (void)phase;
}

void set_precision(Ctx& c, int prec) {
  c.precision = prec;
  c.tc = prec != TN_PREC_C64;
  c.np = (prec == TN_PREC_SPLIT_BF16 || prec == TN_PREC_SPLIT_FP16) ? 4 : 2;
  c.bf16 = prec == TN_PREC_SPLIT_BF16 || prec == TN_PREC_SCALED_BF16;
  c.scaled = prec == TN_PREC_SPLIT_FP16 || prec == TN_PREC_SCALED_FP16 || prec == TN_PREC_SCALED_BF16;
}

tn_status run_step_in(Ctx& c, size_t s, const Geo& g);

// One step in its own precision: the call's, or the per-step override for
// the steps after phase 0 (phase 0 always runs in complex64).
tn_status run_step(Ctx& c, size_t s, const Geo& g) {
  if (!c.step_prec || c.P.steps[s].phase == 0) return run_step_in(c, s, g);
  const int keep = c.precision;
  const bool keep_tc = c.tc, keep_bf16 = c.bf16, keep_scaled = c.scaled;
  const int keep_np = c.np;
  set_precision(c, c.step_prec[s] >= 0 ? (int)c.step_prec[s] : c.call_precision);
  const tn_status r = run_step_in(c, s, g);
  c.precision = keep;
  c.tc = keep_tc;
  c.np = keep_np;
  c.bf16 = keep_bf16;
  c.scaled = keep_scaled;
  return r;
}

tn_status run_step_in(Ctx& c, size_t s, const Geo& g) {
  const Plan& P = c.P;
  Executor& E = c.E;
  const Step& S = P.steps[s];
  GemmDesc d = E.desc[s];
  const float2 *A, *B, *Cc;
  int64_t clo, chi;
  operand(P, E, S.a, S.phase, g, A, d.a_lo, d.a_hi);
  operand(P, E, S.b, S.phase, g, B, d.b_lo, d.b_hi);
  operand(P, E, (int)P.net.leaves.size() + (int)s, S.phase, g, Cc, clo, chi);
  d.c_lo = clo;
  d.c_hi = chi;
  float2* C = const_cast<float2*>(Cc);
  d.units_lo = S.phase == 0 ? 1 : g.gs;
  d.units = S.phase == 0 ? 1 : S.phase == 1 ? g.gs : g.gs * g.gb;
  size_t e0 = 0, e1 = 0;
  if (c.profile && !c.sizing) { tn_status r = c.event(e0); if (r) return r; }
  cudaError_t e;
  int klass = S.klass == SC_VECTOR ? TN_KCLASS_VECTOR : TN_KCLASS_GEMM_SIMT;
  if (S.klass != SC_VECTOR && c.tc && tc_shape_ok(d) && !stream_preferred(d)) klass = TN_KCLASS_GEMM_TC;
  else if (klass == TN_KCLASS_GEMM_SIMT && (!tc_shape_ok(d) || stream_preferred(d)) && vector_shape_ok(d))
    klass = TN_KCLASS_VECTOR;
  // few outputs with a long contracted index: the bandwidth-bound reduction
  const bool reduce = klass == TN_KCLASS_GEMM_SIMT && reduce_shape_ok(d);
  if (reduce) klass = TN_KCLASS_VECTOR;
  if (c.sizing && klass != TN_KCLASS_GEMM_TC) return TN_OK;
  if (reduce) e = launch_reduce(A, B, C, d, c.st);
  else if (klass == TN_KCLASS_VECTOR) {
    VecOut o{};
    e = cudaSuccess;
    if (s < c.max_out.size() && c.max_out[s]) {
      o.maxbits = c.mc_all + s * c.U;
      e = cudaMemsetAsync(o.maxbits, 0, c.U * sizeof(unsigned), c.st);
    }
    if (s < c.planes_out.size() && c.planes_out[s]) {
      // split planes for a tensor-core consumer (unscaled formats only)
      o.mode = 2;
      o.bf16 = c.bf16 ? 1 : 0;
      o.plane = int64_t(1) << (d.nm + d.nn);
    }
    if (e == cudaSuccess) e = launch_vector(A, B, C, d, c.st, o);
  }
  else if (klass == TN_KCLASS_GEMM_TC) {
    const int L = (int)P.net.leaves.size();
    PlaneOperand pa{}, pb{};
    const bool a_in = S.a >= L && c.planes_out[S.a - L] && planes_in_place(A, d, false, c.np, pa);
    const bool b_in = S.b >= L && c.planes_out[S.b - L] && planes_in_place(B, d, true, c.np, pb);
    if ((S.a >= L && c.planes_out[S.a - L] && !a_in) || (S.b >= L && c.planes_out[S.b - L] && !b_in))
      return fail(TN_EINVAL, "step %zu: internal error, operand planes do not match the step's view", s);
    const int64_t need_a = a_in ? 0 : split_scratch_elems(d, false, c.np);
    const int64_t need = need_a + (b_in ? 0 : split_scratch_elems(d, true, c.np));
    if (c.sizing) {
      c.scratch_need = std::max(c.scratch_need, need);
      return TN_OK;
    }
    if (need > E.scratch_cap) return fail(TN_EINVAL, "step %zu: internal error, operand scratch not sized", s);
    for (auto& t : E.tuned)
      if (t.precision == c.precision && t.step == (int)s) {
        d.tile_n = t.tile_n;
        d.group_m = t.group_m;
        d.persistent = t.persistent;
      }
    ScaleIO sio{};
    e = cudaSuccess;
    const int64_t U = c.U;
    // a streaming producer already recorded its output's maxima for the split
    auto recorded = [&](int x) { return x >= L && x - L < (int)c.max_out.size() && c.max_out[x - L]; };
    if (!a_in) {
      const bool ready = c.scaled && recorded(S.a);
      unsigned* mx = ready ? c.mc_all + (S.a - L) * U : c.mb[0];
      if (c.scaled && !ready) e = cudaMemsetAsync(c.mb[0], 0, U * sizeof(unsigned), c.st);
      if (e == cudaSuccess)
        e = split_operand(A, d, false, c.bf16, c.np, c.scaled, mx, c.es[0], c.ms[0], E.scratch, pa, c.st, ready);
      c.launches += c.scaled && !ready ? 2 : 1;
      sio.ea = c.es[0];
      sio.ma = c.ms[0];
    } else {
      sio.ea = c.ec_all + (S.a - L) * U;
      sio.ma = reinterpret_cast<const float*>(c.mc_all + (S.a - L) * U);
    }
    if (!b_in) {
      const bool ready = c.scaled && recorded(S.b);
      unsigned* mx = ready ? c.mc_all + (S.b - L) * U : c.mb[1];
      if (e == cudaSuccess && c.scaled && !ready) e = cudaMemsetAsync(c.mb[1], 0, U * sizeof(unsigned), c.st);
      if (e == cudaSuccess)
        e = split_operand(B, d, true, c.bf16, c.np, c.scaled, mx, c.es[1], c.ms[1], E.scratch + need_a, pb, c.st,
                          ready);
      c.launches += c.scaled && !ready ? 2 : 1;
      sio.eb = c.es[1];
      sio.mb = c.ms[1];
    } else {
      sio.eb = c.ec_all + (S.b - L) * U;
      sio.mb = reinterpret_cast<const float*>(c.mc_all + (S.b - L) * U);
    }
    if (!c.scaled) sio = ScaleIO{};
    else {
      if (c.planes_out[s]) {
        if (e == cudaSuccess) e = cudaMemsetAsync(c.mc_all + s * U, 0, U * sizeof(unsigned), c.st);
        sio.ec = c.ec_all + s * U;
        sio.mc = c.mc_all + s * U;
      }
      sio.flag = S.phase == 1 ? c.flag1 : c.flag2;
      sio.flag_by_lo = S.phase == 1;
    }
    if (c.profile && e == cudaSuccess && need > 0) {
      // the operand split and the GEMM are timed as separate classes
      size_t em = 0;
      tn_status r = c.event(em);
      if (r) return r;
      const double K = std::ldexp(1.0, d.nk), kp = K;
      const double nza = (d.a_lo ? d.units_lo : 1.0) * (d.a_hi ? (double)d.units / d.units_lo : 1.0);
      const double nzb = (d.b_lo ? d.units_lo : 1.0) * (d.b_hi ? (double)d.units / d.units_lo : 1.0);
      const double per = 8.0 + 2.0 * c.np;  // bytes read + written per complex element
      const double bytes = (a_in ? 0.0 : std::ldexp(1.0, d.nm) * (8.0 * K + 2.0 * c.np * kp) * nza) +
                           (b_in ? 0.0 : std::ldexp(1.0, d.nn) * (8.0 * K + 2.0 * c.np * kp) * nzb);
      (void)per;
      c.recs.push_back({TN_KCLASS_SPLIT, 0.0, bytes, e0, (int)s, d.nm, d.nn, d.nk, d.units, 0,
                        (a_in ? 0 : 1) | (b_in ? 0 : 2), 0, 0, 0});
      e0 = em;
    }
    if (e == cudaSuccess && c.tuning) {
      // autotuner: time each tile choice once (every candidate writes the same
      // result; the last launch below leaves it in place) and keep the fastest
      const int def_n = d.nn >= 7 ? 128 : (1 << d.nn);
      float best = 1e30f;
      int bt = 0, bg = 0, bp = 0;
      for (int tn : {128, 64}) {
        if (tn > def_n) continue;
        for (int cand = 0; cand < 6; ++cand) {
          const int gm = (cand % 3 == 0) ? 8 : (cand % 3 == 1) ? 16 : 32;
          const int pers = cand < 3 ? 1 : 2;
          GemmDesc dc = d;
          dc.tile_n = tn;
          dc.group_m = gm;
          dc.persistent = pers;
          cudaEvent_t t0, t1;
          cudaEventCreate(&t0);
          cudaEventCreate(&t1);
          cudaEventRecord(t0, c.st);
          e = launch_gemm_tma(pa, pb, C, c.planes_out[s] != 0, dc, c.bf16, sio, E.err, c.st);
          cudaEventRecord(t1, c.st);
          cudaEventSynchronize(t1);
          float ms = 0;
          cudaEventElapsedTime(&ms, t0, t1);
          cudaEventDestroy(t0);
          cudaEventDestroy(t1);
          if (e != cudaSuccess) break;
          if (ms < best) { best = ms; bt = tn; bg = gm; bp = pers; }
        }
      }
      E.tuned.push_back({c.precision, (int)s, bt, bg, bp});
      d.tile_n = bt;
      d.group_m = bg;
      d.persistent = bp;
    }
    if (e == cudaSuccess) e = launch_gemm_tma(pa, pb, C, c.planes_out[s] != 0, d, c.bf16, sio, E.err, c.st);
  }
  else e = launch_gemm_simt(A, B, C, d, c.st);
  ++c.launches;
  if (e != cudaSuccess) return fail(TN_ECUDA, "step %zu launch: %s", s, cudaGetErrorString(e));
  if (c.profile) {
    tn_status r = c.event(e1);
    if (r) return r;
    const double M = std::ldexp(1.0, d.nm), N = std::ldexp(1.0, d.nn), K = std::ldexp(1.0, d.nk);
    const double U = d.units;
    auto distinct = [&](int64_t lo, int64_t hi) {
      return (lo ? (double)d.units_lo : 1.0) * (hi ? U / d.units_lo : 1.0);
    };
    double bytes = 8.0 * (M * K * distinct(d.a_lo, d.a_hi) + K * N * distinct(d.b_lo, d.b_hi) + M * N * U);
    // diagnostics: C's unit-stride index (row bit i -> i, column bit j -> 100 + j), plane output,
    // 16-column vector stores, which operands vary with the lo / hi unit index
    // C's four fastest indices: row bit i -> i, column bit j -> 100 + j (base-1000 digits)
    long long cfast = 0;
    for (int q = 3; q >= 0; --q) {
      int who = 999;
      for (int i = 0; i < d.nm; ++i) if (d.cm[i] == (1 << q)) who = i;
      for (int j = 0; j < d.nn; ++j) if (d.cn[j] == (1 << q)) who = 100 + j;
      cfast = cfast * 1000 + who;
    }
    const int n16 = d.nn >= 4 && d.cn[0] == 1 && d.cn[1] == 2 && d.cn[2] == 4 && d.cn[3] == 8;
    const int ulo = (d.a_lo ? 1 : 0) | (d.b_lo ? 2 : 0), uhi = (d.a_hi ? 1 : 0) | (d.b_hi ? 2 : 0);
    c.recs.push_back({klass, 8.0 * M * N * K * U, bytes, e0, (int)s, d.nm, d.nn, d.nk, d.units, cfast,
                      (int)(s < c.planes_out.size() && c.planes_out[s]), n16, ulo, uhi});
  }
  return TN_OK;
}

tn_status run_misc(Ctx& c, cudaError_t e, const char* what) {
  ++c.launches;
  if (e != cudaSuccess) return fail(TN_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
  return TN_OK;
}

}  // namespace

static tn_status contract_core(Plan& P, const uint64_t* bits, int64_t nb, double* out, const tn_exec_opts& o,
                               tn_report* rep, bool clear_out, int flags = 3);

tn_status contract_amplitudes(Plan& P, const uint64_t* bits, int64_t nb, double* out, const tn_exec_opts& o,
                              tn_report* rep) {
  return contract_core(P, bits, nb, out, o, rep, true);
}

tn_status contract_amplitudes_ex(Plan& P, const uint64_t* bits, int64_t nb, double* out, const tn_exec_opts& o,
                                 tn_report* rep, bool clear_out, int flags) {
  return contract_core(P, bits, nb, out, o, rep, clear_out, flags);
}

int64_t executor_bytes(const Plan& P) {
  const Executor* E = P.exec;
  if (!E) return 0;
  return 8 * (E->sarena_cap + E->parena_cap + P.invariant_elems + P.leaf_store_elems) + 2 * E->scratch_cap +
         E->spool_cap;
}

static tn_status contract_core(Plan& P, const uint64_t* bits, int64_t nb, double* out, const tn_exec_opts& o,
                               tn_report* rep, bool clear_out, int flags) {
  const int n = P.net.n;
  const int k = (int)P.net.open_qubits.size();
  const int words = std::max(1, (n + 63) / 64);
  const int64_t S_all = num_slice_ids(P);
  const int64_t s_begin = o.slice_begin;
  const int64_t ns = o.slice_count < 0 ? S_all - s_begin : o.slice_count;
  if (s_begin < 0 || s_begin > S_all || ns < 0 || s_begin + ns > S_all)
    return fail(TN_EINVAL, "tn_contract_amplitudes: slice range [%lld, %lld) outside [0, %lld)", (long long)s_begin,
                (long long)(s_begin + ns), (long long)S_all);
  cudaStream_t st = (cudaStream_t)o.stream;
  if (!P.exec) {
    P.exec = new Executor();
    tn_status e = setup(P, *P.exec);
    if (e != TN_OK) { destroy_executor(P.exec); P.exec = nullptr; return e; }
  }
  Executor& E = *P.exec;
  const int64_t nout = nb << k;
  // the precision of each step after phase 0 (the call's unless overridden)
  auto prec_of = [&](size_t s) {
    return o.step_precision && o.step_precision[s] >= 0 ? (int)o.step_precision[s] : (int)o.precision;
  };
  auto is_scaled = [](int pr) {
    return pr == TN_PREC_SPLIT_FP16 || pr == TN_PREC_SCALED_FP16 || pr == TN_PREC_SCALED_BF16;
  };
  bool scaled = is_scaled(o.precision), any_tc = o.precision != TN_PREC_C64;
  if (o.step_precision) {
    scaled = any_tc = false;
    for (size_t s = 0; s < P.steps.size(); ++s)
      if (P.steps[s].phase != 0) {
        scaled |= is_scaled(prec_of(s));
        any_tc |= prec_of(s) != TN_PREC_C64;
      }
  }

  // ---- group geometry: Gb bitstrings x Gs slices per launch
  const int64_t Se = P.slice_arena_elems, Pe = P.unit_arena_elems;
  int64_t Gb = std::max<int64_t>(1, std::min<int64_t>(nb, 256));
  int64_t Gs = o.units_per_group;
  if (Gs <= 0) {
    size_t freeb = 0, totb = 0;
    CK(cudaMemGetInfo(&freeb, &totb));
    double have = (double)(E.sarena_cap + E.parena_cap) * 8.0;
    double budget = std::min<double>((double)freeb * 0.6 + have, 120.0 * (1ull << 30));
    Gs = (int64_t)(budget / (8.0 * ((double)Se + (double)Gb * Pe)));
    while (Gs < 1 && Gb > 1) {  // not even one slice fits with Gb bitstrings: shrink Gb
      Gb = std::max<int64_t>(1, Gb / 2);
      Gs = (int64_t)(budget / (8.0 * ((double)Se + (double)Gb * Pe)));
    }
    Gs = std::min<int64_t>(Gs, 1024);
  }
  Gs = std::max<int64_t>(1, std::min<int64_t>(Gs, std::max<int64_t>(ns, 1)));
  Gs = std::min<int64_t>(Gs, 65535 / Gb);
  if (Gs < 1) return fail(TN_EINVAL, "tn_contract_amplitudes: launch geometry does not fit");
  // captured launch sequences hold the addresses of the arenas, the scale
  // pool and the operand scratch: replacing any of them invalidates them all
  auto drop_graphs = [&]() {
    for (auto& gr : E.graphs) cudaGraphExecDestroy(gr.exec);
    E.graphs.clear();
  };
  auto grow = [&](float2*& p, int64_t& cap, int64_t need) -> tn_status {
    if (cap >= need) return TN_OK;
    drop_graphs();
    cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t ae = dev_alloc(&p, (size_t)need * sizeof(float2));
    if (ae != cudaSuccess) {
      cudaGetLastError();
      return fail(TN_EHBM, "tn_contract_amplitudes: %lld-byte arena does not fit in device memory",
                  (long long)(need * 8));
    }
    cap = need;
    return TN_OK;
  };
  tn_status gs_ = grow(E.sarena, E.sarena_cap, Gs * Se);
  if (gs_ != TN_OK) return gs_;
  gs_ = grow(E.parena, E.parena_cap, Gs * Gb * Pe);
  if (gs_ != TN_OK) return gs_;

  const uint64_t* d_bits = bits;
  double2* d_acc = (double2*)out;
  if (!o.device_io) {
    if (E.bits_cap < nb * words) {
      cudaFree(E.bits);
      E.bits = nullptr;
      E.bits_cap = 0;
      CK(dev_alloc(&E.bits, std::max<int64_t>(nb * words, 1) * sizeof(uint64_t)));
      E.bits_cap = nb * words;
    }
    if (E.acc_cap < nout) {
      cudaFree(E.acc);
      E.acc = nullptr;
      E.acc_cap = 0;
      CK(dev_alloc(&E.acc, std::max<int64_t>(nout, 1) * sizeof(double2)));
      E.acc_cap = nout;
    }
    d_bits = E.bits;
    d_acc = E.acc;
  }
  Ctx c(P, E, st, o.profile != 0);
  set_precision(c, o.precision);
  c.tc = any_tc;
  c.scaled = scaled;
  c.step_prec = o.step_precision;
  c.call_precision = o.precision;
  c.U = Gs * Gb;
  c.planes_out.assign(P.steps.size(), 0);
  const bool handover = o.handover == 1 || (o.handover == 0 && kHandoverDefault[o.precision]);
  auto handover_of = [&](int pr) { return o.handover == 1 || (o.handover == 0 && kHandoverDefault[pr]); };
  if (c.tc) {
    // A step whose consumer also runs on the tensor cores, in the same
    // precision, hands its output over as 16-bit planes laid out for that
    // consumer (no separate split pass).
    const int L = (int)P.net.leaves.size();
    std::vector<char> tc(P.steps.size(), 0);
    for (size_t s = 0; s < P.steps.size(); ++s)
      tc[s] = P.steps[s].klass != SC_VECTOR && tc_shape_ok(E.desc[s]) && !stream_preferred(E.desc[s]) &&
              prec_of(s) != TN_PREC_C64;
    for (size_t t = 0; t < P.steps.size(); ++t) {
      if (!tc[t] || !handover_of(prec_of(t))) continue;
      const Step& S = P.steps[t];
      const int np_t = (prec_of(t) == TN_PREC_SPLIT_BF16 || prec_of(t) == TN_PREC_SPLIT_FP16) ? 4 : 2;
      for (int role = 0; role < 2; ++role) {
        const int x = role ? S.b : S.a;
        if (x < L) continue;
        const int p = x - L;
        PlaneOperand probe{};
        if (P.steps[p].phase == 0 || prec_of(p) != prec_of(t) ||
            !planes_in_place(nullptr, E.desc[t], role == 1, np_t, probe))
          continue;
        // A streaming producer writes split planes too, in an unscaled format
        // (split bf16).  In a scaled one the exponents need the unit's maxima
        // first: a second pass over the input, plus four 2-byte stores per
        // value, cost as much as the split pass they replace (measured on the
        // 8x8 plan), so there the producer records the maxima for the split.
        const GemmDesc& dp = E.desc[p];
        const bool streams = P.steps[p].klass == SC_VECTOR ||
                             ((!tc_shape_ok(dp) || stream_preferred(dp)) && vector_shape_ok(dp));
        if (tc[p] || (streams && np_t == 4 && !is_scaled(prec_of(t)))) c.planes_out[p] = 1;
      }
    }
    // A streaming step (complex64 output) feeding a tensor-core step in a
    // scaled format records its output's maxima as it writes, and the split
    // pass skips its maximum pass.
    c.max_out.assign(P.steps.size(), 0);
    for (size_t t = 0; t < P.steps.size(); ++t) {
      if (!tc[t] || !is_scaled(prec_of(t))) continue;
      const Step& S = P.steps[t];
      for (int x : {S.a, S.b}) {
        if (x < L) continue;
        const int p = x - L;
        const GemmDesc& dp = E.desc[p];
        const bool streams = P.steps[p].klass == SC_VECTOR ||
                             ((!tc_shape_ok(dp) || stream_preferred(dp)) && vector_shape_ok(dp));
        if (P.steps[p].phase != 0 && !c.planes_out[p] && streams) c.max_out[p] = 1;
      }
    }
  }
  if (scaled) {
    // scale pool: ec, mc per step; e, m, maxbits per split role; flags
    const int64_t ns_ = (int64_t)P.steps.size();
    const int64_t need = 8 * ns_ * c.U + 2 * 12 * c.U + 4 * (Gs + c.U) + 256;
    if (E.spool_cap < need) {
      drop_graphs();
      cudaFree(E.spool);
      E.spool = nullptr;
      E.spool_cap = 0;
      CK(dev_alloc(&E.spool, need));
      E.spool_cap = need;
    }
    uint8_t* q = E.spool;
    c.ec_all = (int*)q;                      q += 4 * ns_ * c.U;
    c.mc_all = (unsigned*)q;                 q += 4 * ns_ * c.U;
    for (int r = 0; r < 2; ++r) {
      c.es[r] = (int*)q;                     q += 4 * c.U;
      c.ms[r] = (float*)q;                   q += 4 * c.U;
      c.mb[r] = (unsigned*)q;                q += 4 * c.U;
    }
    c.flag1 = (int*)q;                       q += 4 * Gs;
    c.flag2 = (int*)q;
  }
  if (clear_out) CK(cudaEventRecord(E.ev0, st));  // a nested recompute call is timed by its caller
  if (!o.device_io && nb > 0)
    CK(cudaMemcpyAsync((void*)d_bits, bits, nb * words * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  if (nout > 0 && clear_out) CK(cudaMemsetAsync(d_acc, 0, nout * sizeof(double2), st));
  if (scaled && (flags & 1)) CK(cudaMemsetAsync(E.nflagged, 0, sizeof(unsigned long long), st));
  Geo g;
  if (!E.inv_ready) {
    // invariant steps once, always in complex64 so that any later precision
    // can use them; with a shared stem, once for every plan of the circuit
    std::unique_lock<std::mutex> lk;
    if (E.stem) lk = std::unique_lock<std::mutex>(E.stem->mu);
    if (E.stem && E.stem->inv_ready) {
      CK(cudaStreamWaitEvent(st, E.stem->ready, 0));
      E.stem_reused = true;
    } else {
      const int keep = c.precision;
      const bool keep_tc = c.tc;
      c.precision = TN_PREC_C64;
      c.tc = false;
      for (size_t s = 0; s < P.steps.size(); ++s)
        if (P.steps[s].phase == 0) {
          tn_status r = run_step(c, s, g);
          if (r != TN_OK) return r;
        }
      c.precision = keep;
      c.tc = keep_tc;
      if (E.stem) {
        CK(cudaEventRecord(E.stem->ready, st));
        E.stem->inv_ready = true;
      }
    }
    E.inv_ready = true;
  }
  const int L = (int)P.net.leaves.size();
  const int root_id = L == 1 ? 0 : L + (int)P.steps.size() - 1;
  // operand scratch for the tensor-core steps, sized before any launch so that
  // the launch sequences allocate nothing (and can be captured as graphs)
  if (c.tc && nb > 0) {
    c.sizing = true;
    Geo gz;
    gz.gs = (int)std::min<int64_t>(Gs, std::max<int64_t>(ns, 1));
    gz.gb = (int)std::min<int64_t>(Gb, nb);
    for (size_t s = 0; s < P.steps.size(); ++s)
      if (P.steps[s].phase != 0) {
        tn_status r = run_step(c, s, gz);
        if (r != TN_OK) return r;
      }
    c.sizing = false;
    if (c.scratch_need > E.scratch_cap) {
      drop_graphs();
      cudaFree(E.scratch);
      E.scratch = nullptr;
      E.scratch_cap = 0;
      if (dev_alloc(&E.scratch, (size_t)c.scratch_need * sizeof(uint16_t)) != cudaSuccess) {
        cudaGetLastError();
        return fail(TN_EHBM, "tn_contract_amplitudes: %lld bytes of operand planes do not fit",
                    (long long)(c.scratch_need * 2));
      }
      E.scratch_cap = c.scratch_need;
    }
  }
  // autotuner: the first group of a precision times the tile choices
  if (c.tc && o.autotune) {
    if (!E.tune_loaded) {
      E.tune_loaded = true;
      if (const char* path = getenv("TN_AUTOTUNE_CACHE")) {
        if (FILE* f = fopen(path, "r")) {
          unsigned long long h;
          int pr, st_, tn, gm;
          int pe;
          while (fscanf(f, "%llx %d %d %d %d %d", &h, &pr, &st_, &tn, &gm, &pe) == 6)
            if (h == P.hash) E.tuned.push_back({pr, st_, tn, gm, pe});
          fclose(f);
        }
      }
    }
    bool have = false;
    for (auto& t : E.tuned) have |= t.precision == c.precision;
    c.tuning = !have;
  }
  // (stream capture needs an explicit stream: the legacy default stream cannot be captured)
  const bool graphs = o.use_graph && st != nullptr && !o.profile && !(scaled && o.test_flag_every > 0) &&
                      !o.step_precision;
  // One launch sequence (the slice-only steps of a group, or the per-unit
  // steps of a group and its accumulation), replayed from a graph when allowed.
  auto sequence = [&](int phase, const Geo& gg) -> tn_status {
    auto body = [&]() -> tn_status {
      if (phase == 1) {
        if (scaled) CK(cudaMemsetAsync(c.flag1, 0, Gs * sizeof(int), st));
        if (E.ngather1) {
          tn_status r = run_misc(c, launch_gather(E.store, E.sarena, Se, E.gather, E.ngather1, E.gslot, gg.gs, st),
                                 "gather");
          if (r) return r;
        }
      } else {
        if (scaled) CK(cudaMemsetAsync(c.flag2, 0, c.U * sizeof(int), st));
        if (E.ngather2) {
          tn_status r = run_misc(
              c, launch_gather(E.store, E.parena, Pe, E.gather + E.ngather1, E.ngather2, E.gslot + 1, gg.gs * gg.gb, st),
              "gather");
          if (r) return r;
        }
      }
      for (size_t s = 0; s < P.steps.size(); ++s)
        if (P.steps[s].phase == phase) {
          tn_status r = run_step(c, s, gg);
          if (r != TN_OK) return r;
        }
      if (phase == 2) {
        const float2* root;
        int64_t rlo, rhi;
        operand(P, E, root_id, 2, gg, root, rlo, rhi);
        tn_status r = run_misc(c,
                               launch_accumulate(root, rlo, rhi, E.perm, (int)P.root_perm.size(), E.gslot + 1, gg.gb,
                                                 scaled ? c.flag1 : nullptr, scaled ? c.flag2 : nullptr, E.flagged,
                                                 E.nflagged, kFlaggedCap, st),
                               "accumulate");
        if (r) return r;
      }
      return TN_OK;
    };
    if (!graphs || c.tuning) return body();
    for (auto& gr : E.graphs)
      if (gr.phase == phase && gr.precision == c.precision && gr.handover == (int)handover && gr.gs == gg.gs &&
          gr.gb == (phase == 2 ? gg.gb : 1)) {
        CK(cudaGraphLaunch(gr.exec, st));
        c.launches += gr.kernels;
        return TN_OK;
      }
    const int64_t before = c.launches;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    tn_status r = body();
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (r != TN_OK) {
      if (graph) cudaGraphDestroy(graph);
      return r;
    }
    if (ce != cudaSuccess) return fail(TN_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(TN_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    E.graphs.push_back({phase, c.precision, (int)handover, gg.gs, phase == 2 ? gg.gb : 1, exec, c.launches - before});
    CK(cudaGraphLaunch(exec, st));
    return TN_OK;
  };
  for (int64_t s0 = s_begin; s0 < s_begin + ns && nb > 0; s0 += Gs) {
    g.gs = (int)std::min<int64_t>(Gs, s_begin + ns - s0);
    g.gb = 1;
    GroupInfo gi{};
    gi.slice0 = s0;
    gi.b0 = 0;
    gi.nslice = g.gs;
    gi.nb = 1;
    gi.words = words;
    gi.units = g.gs;
    gi.bits = d_bits;
    gi.acc = d_acc;
    {
      tn_status r = run_misc(c, launch_set_group(E.gslot, gi, st), "set_group");
      if (r) return r;
    }
    if (scaled && o.test_flag_every > 0) {
      // host-side injection of filter flags (tests of the recompute / discard paths)
      CK(cudaMemsetAsync(c.flag1, 0, Gs * sizeof(int), st));
      std::vector<int> f(g.gs);
      for (int i = 0; i < g.gs; ++i) f[i] = ((s0 + i) % o.test_flag_every) == 0;
      tn_status r = sequence(1, g);
      if (r) return r;
      CK(cudaMemcpyAsync(c.flag1, f.data(), g.gs * sizeof(int), cudaMemcpyHostToDevice, st));
      CK(cudaStreamSynchronize(st));
    } else {
      tn_status r = sequence(1, g);
      if (r) return r;
    }
    for (int64_t b0 = 0; b0 < nb; b0 += Gb) {
      g.gb = (int)std::min<int64_t>(Gb, nb - b0);
      gi.b0 = b0;
      gi.nb = g.gb;
      gi.units = g.gs * g.gb;
      tn_status r = run_misc(c, launch_set_group(E.gslot + 1, gi, st), "set_group");
      if (r) return r;
      r = sequence(2, g);
      if (r) return r;
    }
    if (c.tuning) {
      c.tuning = false;
      if (const char* path = getenv("TN_AUTOTUNE_CACHE")) {
        if (FILE* f = fopen(path, "a")) {
          for (auto& t : E.tuned)
            if (t.precision == c.precision)
              fprintf(f, "%llx %d %d %d %d %d\n", (unsigned long long)P.hash, t.precision, t.step, t.tile_n,
                      t.group_m, t.persistent);
          fclose(f);
        }
      }
    }
  }
  // ---- the filter: units flagged in a scaled precision are recomputed in
  // complex64 (policy 0) or left out and counted (policy 1)
  int64_t nflag = 0, recomputed = 0, discarded = 0;
  if (scaled && nb > 0 && (flags & 2)) {
    unsigned long long hn = 0;
    CK(cudaMemcpyAsync(&hn, E.nflagged, sizeof(hn), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    nflag = (int64_t)hn;
    if (nflag > kFlaggedCap)
      return fail(TN_EOVERFLOW, "tn_contract_amplitudes: %lld units flagged (more than %d listed)", (long long)nflag,
                  kFlaggedCap);
    if (nflag > 0) {
      std::vector<int64_t> list(nflag);
      CK(cudaMemcpy(list.data(), E.flagged, nflag * sizeof(int64_t), cudaMemcpyDeviceToHost));
      if (o.overflow_policy == 1) {
        discarded = nflag;
      } else {
        for (int64_t f : list) {
          const int64_t b = f >> 32, s = f & 0xffffffffll;
          tn_exec_opts r = o;
          r.precision = TN_PREC_C64;
          r.step_precision = nullptr;
          r.device_io = 1;
          r.slice_begin = s;
          r.slice_count = 1;
          r.units_per_group = 1;
          r.profile = 0;
          tn_status rs = contract_core(P, d_bits + b * words, 1, (double*)(d_acc + b * ((int64_t)1 << k)), r,
                                       nullptr, false);
          if (rs != TN_OK) return rs;
          ++recomputed;
        }
      }
    }
  }
  if (!o.device_io && nout > 0) CK(cudaMemcpyAsync(out, d_acc, nout * sizeof(double2), cudaMemcpyDeviceToHost, st));
  if (!clear_out) return TN_OK;
  CK(cudaEventRecord(E.ev1, st));
  if (!o.device_io || rep) {
    CK(cudaEventSynchronize(E.ev1));
    int herr = 0;
    CK(cudaMemcpy(&herr, E.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) {
      CK(cudaMemset(E.err, 0, sizeof(int)));
      return fail(TN_ETIMEOUT, "tn_contract_amplitudes: a tensor-core pipeline wait expired (code %d)", herr);
    }
  }
  if (rep) {
    std::memset(rep, 0, sizeof *rep);
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, E.ev0, E.ev1));
    rep->device_ms = ms;
    rep->units = nb * ns;
    const double shared = P.cmac_slice_only, per = P.cmac_per_slice;
    rep->flops = 8.0 * ((double)ns * shared + (double)nb * ns * (per - shared));
    rep->flops_equivalent = 8.0 * per * (double)nb * ns;
    rep->kernel_launches = c.launches;
    rep->flagged_units = nflag;
    rep->discarded_units = discarded;
    // TN_PROFILE_STEPS=1: per-step breakdown of the timed launches on stderr,
    // one JSON object per step, slowest first.  c_fastest lists C's four
    // fastest indices (stride 8, 4, 2, 1) as three-digit codes: row bit i ->
    // i, column bit j -> 100 + j, none -> 999.
    struct StepAgg { int step = 0, klass = 0, nm = 0, nn = 0, nk = 0, launches = 0, planes = 0, n16 = 0, ulo = 0, uhi = 0; long long cfast = 0; int64_t units = 0; double ms = 0, flops = 0; };
    std::map<int, StepAgg> per_step;
    const bool by_step = getenv("TN_PROFILE_STEPS") != nullptr;
    for (auto& r : c.recs) {
      float t = 0;
      CK(cudaEventElapsedTime(&t, E.pev[r.ev], E.pev[r.ev + 1]));
      rep->class_ms[r.klass] += t;
      rep->class_launches[r.klass] += 1;
      rep->class_flops[r.klass] += r.flops;
      rep->class_bytes[r.klass] += r.bytes;
      if (by_step) {
        // a step's operand split pass is listed apart from its GEMM
        StepAgg& a = per_step[r.klass == TN_KCLASS_SPLIT ? -1 - r.step : r.step];
        a.step = r.step;
        a.klass = r.klass;
        a.nm = r.nm;
        a.nn = r.nn;
        a.nk = r.nk;
        a.cfast = r.cfast;
        a.planes = r.planes;
        a.n16 = r.n16;
        a.ulo = r.ulo;
        a.uhi = r.uhi;
        a.units += r.units;
        a.launches += 1;
        a.ms += t;
        a.flops += r.flops;
      }
    }
    if (by_step) {
      std::vector<std::pair<int, StepAgg>> v(per_step.begin(), per_step.end());
      std::sort(v.begin(), v.end(), [](const auto& x, const auto& y) { return x.second.ms > y.second.ms; });
      static const char* kname[4] = {"simt", "vector", "tensor", "split"};
      for (auto& [st_i, a] : v)
        fprintf(stderr,
                "{\"step\": %d, \"phase\": %d, \"class\": \"%s\", \"log2_m\": %d, \"log2_n\": %d, "
                "\"log2_k\": %d, \"units\": %lld, \"launches\": %d, \"ms\": %.3f, \"tflops\": %.1f, "
                "\"c_fastest\": \"%012lld\", \"planes_out\": %d, \"vec16\": %d, \"a_b_vary_lo\": %d, "
                "\"a_b_vary_hi\": %d}\n",
                a.step, P.steps[a.step].phase, kname[a.klass & 3], a.nm, a.nn, a.nk, (long long)a.units, a.launches,
                a.ms, a.ms > 0 ? a.flops / (a.ms * 1e9) : 0.0, a.cfast, a.planes, a.n16, a.ulo, a.uhi);
    }
  }
  (void)recomputed;
  return TN_OK;
}

}  // namespace tn

using namespace tn;

extern "C" tn_status tn_contract_amplitudes(tn_plan_t* p, const uint64_t* bits, int64_t nb, double* out,
                                            const tn_exec_opts* opts, tn_report* rep) {
  if (!p) return fail(TN_EINVAL, "tn_contract_amplitudes: plan is NULL");
  if (nb < 0 || (nb > 0 && (!bits || !out))) return fail(TN_EINVAL, "tn_contract_amplitudes: bad bitstrings/out");
  const int k = (int)p->plan.net.open_qubits.size();
  if (nb > (int64_t(1) << (40 - k)))
    return fail(TN_EINVAL, "tn_contract_amplitudes: %lld bitstrings x 2^%d amplitudes exceed 2^40", (long long)nb, k);
  tn_exec_opts o;
  std::memset(&o, 0, sizeof o);
  o.slice_count = -1;
  if (opts) o = *opts;
  if (o.units_per_group < 0) return fail(TN_EINVAL, "tn_contract_amplitudes: units_per_group < 0");
  if (o.precision < TN_PREC_C64 || o.precision > TN_PREC_SCALED_BF16)
    return fail(TN_EINVAL, "tn_contract_amplitudes: unknown precision %d", o.precision);
  if (o.step_precision)
    for (size_t s = 0; s < p->plan.steps.size(); ++s)
      if (o.step_precision[s] < -1 || o.step_precision[s] > TN_PREC_SCALED_BF16)
        return fail(TN_EINVAL, "tn_contract_amplitudes: step %zu: unknown precision %d", s, (int)o.step_precision[s]);
  return guarded("tn_contract_amplitudes", [&] { return contract_amplitudes(p->plan, bits, nb, out, o, rep); });
}

extern "C" void tn_free_plan(tn_plan_t* p) { delete p; }
