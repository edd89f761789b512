// Executor: runs a plan's step chain over groups of (bitstring, slice) units
// and sums the unit results in FP64 (paper: Sec. "A Customized Parallelization
// Scheme" -- slices are independent sub-tasks; here they are the units of one
// GPU's work instead of MPI processes -- and Sec. "Scaling", global reduction).
//
// Device memory of a plan (allocated on first use, kept until tn_free_plan):
//   leaf store  -- every leaf tensor in complex64, full (fixed indices included)
//   invariant   -- outputs of steps that depend on no fixed index (computed once)
//   unit arena  -- G units x per-unit arena: variant leaf sub-tensors and
//                  variant step outputs at the planner's liveness offsets
//   accumulator -- nb x 2^k complex128
#include <algorithm>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "tn_internal.h"

namespace tn {

struct Executor {
  int device = -1;
  float2* store = nullptr;
  float2* inv = nullptr;
  bool inv_ready = false;
  float2* arena = nullptr;
  int64_t arena_units = 0;
  LeafGather* gather = nullptr;
  int ngather = 0;
  int64_t* perm = nullptr;
  uint64_t* bits = nullptr;
  int64_t bits_cap = 0;
  double2* acc = nullptr;
  int64_t acc_cap = 0;
  std::vector<GemmDesc> desc;  // per step, unit strides filled at launch
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

void destroy_executor(Executor* e) {
  if (!e) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (e->device >= 0) cudaSetDevice(e->device);
  cudaFree(e->store);
  cudaFree(e->inv);
  cudaFree(e->arena);
  cudaFree(e->gather);
  cudaFree(e->perm);
  cudaFree(e->bits);
  cudaFree(e->acc);
  if (e->ev0) cudaEventDestroy(e->ev0);
  if (e->ev1) cudaEventDestroy(e->ev1);
  if (cur >= 0) cudaSetDevice(cur);
  delete e;
}

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t _e = (call);                                                                 \
    if (_e != cudaSuccess) return fail(TN_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__, __LINE__); \
  } while (0)

// Per-bit strides of the GEMM view of one step (see GemmDesc).
void make_gemm_desc(const std::vector<int>& la, const std::vector<int>& lb, const std::vector<int>& lc,
                    GemmDesc& d) {
  std::memset(&d, 0, sizeof d);
  auto stride_in = [](const std::vector<int>& ls, int l) -> int32_t {
    for (size_t p = 0; p < ls.size(); ++p)
      if (ls[p] == l) return int32_t(1) << (ls.size() - 1 - p);
    return -1;
  };
  // walk each operand from its fastest index upward
  for (int p = (int)la.size() - 1; p >= 0; --p) {
    int l = la[p];
    int32_t sb = stride_in(lb, l);
    if (sb < 0) { d.am[d.nm] = stride_in(la, l); d.cm[d.nm] = stride_in(lc, l); ++d.nm; }
    else { d.ak[d.nk] = stride_in(la, l); d.bk[d.nk] = sb; ++d.nk; }
  }
  for (int p = (int)lb.size() - 1; p >= 0; --p) {
    int l = lb[p];
    if (stride_in(la, l) < 0) { d.bn[d.nn] = stride_in(lb, l); d.cn[d.nn] = stride_in(lc, l); ++d.nn; }
  }
}

static tn_status setup(Plan& P, Executor& E) {
  CK(cudaGetDevice(&E.device));
  const Network& N = P.net;
  const int L = (int)N.leaves.size();
  std::vector<float2> h_store(P.leaf_store_elems);
  for (int i = 0; i < L; ++i) {
    const Leaf& lf = N.leaves[i];
    for (size_t e = 0; e < lf.data.size(); ++e)
      h_store[P.leaf_use[i].store_off + e] = make_float2((float)lf.data[e].real(), (float)lf.data[e].imag());
  }
  CK(cudaMalloc(&E.store, std::max<int64_t>(P.leaf_store_elems, 1) * sizeof(float2)));
  CK(cudaMemcpy(E.store, h_store.data(), h_store.size() * sizeof(float2), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&E.inv, P.invariant_elems * sizeof(float2)));
  std::vector<LeafGather> g;
  for (int i = 0; i < L; ++i) {
    const LeafUse& U = P.leaf_use[i];
    if (!U.variant) continue;
    const Leaf& lf = N.leaves[i];
    LeafGather d;
    std::memset(&d, 0, sizeof d);
    if ((int)lf.labels.size() > kMaxLeafRank) return fail(TN_EINVAL, "leaf rank %zu > %d", lf.labels.size(), kMaxLeafRank);
    d.store_off = U.store_off;
    d.dst_off = U.off;
    const int r = (int)lf.labels.size();
    for (int p = 0; p < r; ++p) {
      int32_t st = int32_t(1) << (r - 1 - p);
      if (U.fixed_src[p] == -1) d.kept_stride[d.nkept++] = st;
      else { d.fixed_src[d.nfixed] = U.fixed_src[p]; d.fixed_stride[d.nfixed] = st; ++d.nfixed; }
    }
    g.push_back(d);
  }
  E.ngather = (int)g.size();
  if (!g.empty()) {
    CK(cudaMalloc(&E.gather, g.size() * sizeof(LeafGather)));
    CK(cudaMemcpy(E.gather, g.data(), g.size() * sizeof(LeafGather), cudaMemcpyHostToDevice));
  }
  CK(cudaMalloc(&E.perm, P.root_perm.size() * sizeof(int64_t)));
  CK(cudaMemcpy(E.perm, P.root_perm.data(), P.root_perm.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  E.desc.resize(P.steps.size());
  for (size_t s = 0; s < P.steps.size(); ++s) make_gemm_desc(P.steps[s].la, P.steps[s].lb, P.steps[s].lc, E.desc[s]);
  CK(cudaEventCreate(&E.ev0));
  CK(cudaEventCreate(&E.ev1));
  return TN_OK;
}

// Operand pointer and unit stride of SSA id x.
static void operand(const Plan& P, const Executor& E, int x, const float2*& ptr, int64_t& unit_stride) {
  const int L = (int)P.net.leaves.size();
  if (x < L) {
    const LeafUse& U = P.leaf_use[x];
    if (U.variant) { ptr = E.arena + U.off; unit_stride = P.unit_arena_elems; }
    else { ptr = E.store + U.store_off; unit_stride = 0; }
  } else {
    const Step& S = P.steps[x - L];
    if (S.variant) { ptr = E.arena + S.off_c; unit_stride = P.unit_arena_elems; }
    else { ptr = E.inv + S.off_c; unit_stride = 0; }
  }
}

static tn_status run_step(const Plan& P, Executor& E, size_t s, int units, cudaStream_t st, int64_t& launches) {
  const Step& S = P.steps[s];
  GemmDesc d = E.desc[s];
  const float2 *A, *B;
  operand(P, E, S.a, A, d.a_unit);
  operand(P, E, S.b, B, d.b_unit);
  float2* C = (S.variant ? E.arena : E.inv) + S.off_c;
  d.c_unit = S.variant ? P.unit_arena_elems : 0;
  d.units = S.variant ? units : 1;
  cudaError_t e;
  if (S.klass == SC_VECTOR) e = launch_vector(A, B, C, d, st);
  else e = launch_gemm_simt(A, B, C, d, st);
  ++launches;
  if (e != cudaSuccess) return fail(TN_ECUDA, "step %zu launch: %s", s, cudaGetErrorString(e));
  return TN_OK;
}

tn_status contract_amplitudes(Plan& P, const uint64_t* bits, int64_t nb, double* out, const tn_exec_opts& o,
                              tn_report* rep) {
  if (o.precision != TN_PREC_C64)
    return fail(TN_EINVAL, "tn_contract_amplitudes: precision %d not available in this build", o.precision);
  const int n = P.net.n;
  const int k = (int)P.net.open_qubits.size();
  const int words = std::max(1, (n + 63) / 64);
  const int64_t S_all = int64_t(1) << P.sliced.size();
  const int64_t s0 = o.slice_begin;
  const int64_t ns = o.slice_count < 0 ? S_all - s0 : o.slice_count;
  if (s0 < 0 || s0 > S_all || ns < 0 || s0 + ns > S_all)
    return fail(TN_EINVAL, "tn_contract_amplitudes: slice range [%lld, %lld) outside [0, %lld)", (long long)s0,
                (long long)(s0 + ns), (long long)S_all);
  cudaStream_t st = (cudaStream_t)o.stream;
  if (!P.exec) {
    P.exec = new Executor();
    tn_status e = setup(P, *P.exec);
    if (e != TN_OK) { destroy_executor(P.exec); P.exec = nullptr; return e; }
  }
  Executor& E = *P.exec;
  const int64_t nout = nb << k;
  const int64_t total_units = nb * ns;
  int64_t launches = 0;

  // group size
  int64_t G = o.units_per_group;
  if (G <= 0) {
    size_t freeb = 0, totb = 0;
    CK(cudaMemGetInfo(&freeb, &totb));
    double budget = std::min<double>((double)freeb * 0.5 + (double)E.arena_units * P.unit_arena_elems * 8.0,
                                     96.0 * (1ull << 30));
    G = (int64_t)(budget / (P.unit_arena_elems * 8.0));
    G = std::min<int64_t>(G, 1024);
  }
  G = std::max<int64_t>(1, std::min<int64_t>({G, std::max<int64_t>(total_units, 1), 65535}));
  if (E.arena_units < G) {
    cudaFree(E.arena);
    E.arena = nullptr;
    E.arena_units = 0;
    size_t bytes = (size_t)G * P.unit_arena_elems * sizeof(float2);
    cudaError_t ae = cudaMalloc(&E.arena, bytes);
    if (ae != cudaSuccess) {
      cudaGetLastError();
      return fail(TN_EHBM, "tn_contract_amplitudes: arena of %zu bytes (%lld units) does not fit", bytes, (long long)G);
    }
    E.arena_units = G;
  }
  // bitstrings and accumulator
  const uint64_t* d_bits = bits;
  double2* d_acc = (double2*)out;
  if (!o.device_io) {
    if (E.bits_cap < nb * words) {
      cudaFree(E.bits);
      E.bits = nullptr;
      CK(cudaMalloc(&E.bits, std::max<int64_t>(nb * words, 1) * sizeof(uint64_t)));
      E.bits_cap = nb * words;
    }
    if (E.acc_cap < nout) {
      cudaFree(E.acc);
      E.acc = nullptr;
      CK(cudaMalloc(&E.acc, std::max<int64_t>(nout, 1) * sizeof(double2)));
      E.acc_cap = nout;
    }
    d_bits = E.bits;
    d_acc = E.acc;
  }
  CK(cudaEventRecord(E.ev0, st));
  if (!o.device_io && nb > 0) CK(cudaMemcpyAsync((void*)d_bits, bits, nb * words * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  if (nout > 0) CK(cudaMemsetAsync(d_acc, 0, nout * sizeof(double2), st));
  // invariant steps once
  if (!E.inv_ready) {
    for (size_t s = 0; s < P.steps.size(); ++s)
      if (!P.steps[s].variant) {
        tn_status e = run_step(P, E, s, 1, st, launches);
        if (e != TN_OK) return e;
      }
    E.inv_ready = true;
  }
  const int L = (int)P.net.leaves.size();
  const float2* root;
  int64_t root_stride;
  operand(P, E, L == 1 ? 0 : L + (int)P.steps.size() - 1, root, root_stride);
  for (int64_t u0 = 0; u0 < total_units; u0 += G) {
    GroupInfo gi;
    gi.unit0 = u0;
    gi.slices = ns;
    gi.slice_begin = s0;
    gi.words = words;
    gi.units = (int)std::min<int64_t>(G, total_units - u0);
    cudaError_t e = launch_gather(E.store, E.arena, P.unit_arena_elems, E.gather, E.ngather, d_bits, gi, st);
    ++launches;
    if (e != cudaSuccess) return fail(TN_ECUDA, "gather launch: %s", cudaGetErrorString(e));
    for (size_t s = 0; s < P.steps.size(); ++s)
      if (P.steps[s].variant) {
        tn_status r = run_step(P, E, s, gi.units, st, launches);
        if (r != TN_OK) return r;
      }
    e = launch_accumulate(root, root_stride, E.perm, (int)P.root_perm.size(), d_acc, gi, st);
    ++launches;
    if (e != cudaSuccess) return fail(TN_ECUDA, "accumulate launch: %s", cudaGetErrorString(e));
  }
  if (!o.device_io && nout > 0)
    CK(cudaMemcpyAsync(out, d_acc, nout * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CK(cudaEventRecord(E.ev1, st));
  if (!o.device_io || rep) CK(cudaEventSynchronize(E.ev1));
  if (rep) {
    std::memset(rep, 0, sizeof *rep);
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, E.ev0, E.ev1));
    rep->device_ms = ms;
    rep->units = total_units;
    rep->flops = 8.0 * P.cmac_per_slice * (double)total_units;
    rep->kernel_launches = launches;
  }
  return TN_OK;
}

}  // namespace tn

using namespace tn;

extern "C" tn_status tn_contract_amplitudes(tn_plan_t* p, const uint64_t* bits, int64_t nb, double* out,
                                            const tn_exec_opts* opts, tn_report* rep) {
  if (!p) return fail(TN_EINVAL, "tn_contract_amplitudes: plan is NULL");
  if (nb < 0 || (nb > 0 && (!bits || !out))) return fail(TN_EINVAL, "tn_contract_amplitudes: bad bitstrings/out");
  tn_exec_opts o;
  std::memset(&o, 0, sizeof o);
  o.slice_count = -1;
  if (opts) o = *opts;
  if (o.units_per_group < 0) return fail(TN_EINVAL, "tn_contract_amplitudes: units_per_group < 0");
  if (o.precision < TN_PREC_C64 || o.precision > TN_PREC_SCALED_BF16)
    return fail(TN_EINVAL, "tn_contract_amplitudes: unknown precision %d", o.precision);
  return contract_amplitudes(p->plan, bits, nb, out, o, rep);
}

extern "C" void tn_free_plan(tn_plan_t* p) { delete p; }
