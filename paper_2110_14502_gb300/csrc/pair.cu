// tn_contract_pair: one pairwise contraction on device tensors, through the
// executor's kernels (fused) or as permute -> library GEMM -> permute
// (unfused, the comparison baseline of the microbenchmark).
#include <cublas_v2.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.h"
#include "tn_internal.h"

namespace tn {

static tn_status check_labels(const int32_t* la, int ra, const int32_t* lb, int rb, const int32_t* lc, int rc) {
  auto has = [](const int32_t* l, int r, int x) { return std::find(l, l + r, x) != l + r; };
  auto distinct = [](const int32_t* l, int r) {
    std::vector<int> v(l, l + r);
    std::sort(v.begin(), v.end());
    return std::adjacent_find(v.begin(), v.end()) == v.end();
  };
  if (!distinct(la, ra) || !distinct(lb, rb) || !distinct(lc, rc))
    return fail(TN_EINVAL, "tn_contract_pair: repeated label within a tensor");
  for (int i = 0; i < rc; ++i)
    if (has(la, ra, lc[i]) == has(lb, rb, lc[i]))
      return fail(TN_EINVAL, "tn_contract_pair: output label %d must appear in exactly one operand", lc[i]);
  for (int i = 0; i < ra; ++i)
    if (!has(lb, rb, la[i]) && !has(lc, rc, la[i]))
      return fail(TN_EINVAL, "tn_contract_pair: label %d of A is neither contracted nor in C", la[i]);
  for (int i = 0; i < rb; ++i)
    if (!has(la, ra, lb[i]) && !has(lc, rc, lb[i]))
      return fail(TN_EINVAL, "tn_contract_pair: label %d of B is neither contracted nor in C", lb[i]);
  return TN_OK;
}

static cublasHandle_t cublas_handle(int dev) {
  static std::mutex mu;
  static std::vector<cublasHandle_t> hs;
  std::lock_guard<std::mutex> g(mu);
  if ((int)hs.size() <= dev) hs.resize(dev + 1, nullptr);
  if (!hs[dev] && cublasCreate(&hs[dev]) != CUBLAS_STATUS_SUCCESS) hs[dev] = nullptr;
  return hs[dev];
}

// Device state of the tensor-core algorithms, one per device: the kernels'
// error word and a grow-only buffer for the operand planes.  A call holds the
// mutex until its kernel has finished, so calls on one device are serialised
// and the buffer is never in use by two calls at once.
struct PairDevState {
  int* err = nullptr;
  void* scratch = nullptr;
  size_t bytes = 0;
};
static std::mutex g_pair_mu;
static std::vector<PairDevState> g_pair_state;

static tn_status pair_state(size_t need, PairDevState*& out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(TN_ECUDA, "tn_contract_pair: cudaGetDevice failed");
  if ((int)g_pair_state.size() <= dev) g_pair_state.resize(dev + 1);
  PairDevState& st = g_pair_state[dev];
  if (!st.err) {
    if (cudaMalloc(&st.err, sizeof(int)) != cudaSuccess) return fail(TN_ECUDA, "tn_contract_pair: error word");
    if (cudaMemset(st.err, 0, sizeof(int)) != cudaSuccess) return fail(TN_ECUDA, "tn_contract_pair: error word");
  }
  if (need > st.bytes) {
    cudaFree(st.scratch);  // the previous call on this device has finished
    st.scratch = nullptr;
    st.bytes = 0;
    if (cudaMalloc(&st.scratch, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(TN_EHBM, "tn_contract_pair: operand planes do not fit");
    }
    st.bytes = need;
  }
  out = &st;
  return TN_OK;
}

static tn_status unfused(const float2* A, const float2* B, float2* Cp, const GemmDesc& d, cudaStream_t st) {
  const int64_t M = int64_t(1) << d.nm, N = int64_t(1) << d.nn, K = int64_t(1) << d.nk;
  float2 *Ap = nullptr, *Bp = nullptr, *Cg = nullptr;
  auto cleanup = [&]() {
    if (Ap) cudaFreeAsync(Ap, st);
    if (Bp) cudaFreeAsync(Bp, st);
    if (Cg) cudaFreeAsync(Cg, st);
  };
  if (cudaMallocAsync(&Ap, M * K * sizeof(float2), st) != cudaSuccess ||
      cudaMallocAsync(&Bp, K * N * sizeof(float2), st) != cudaSuccess ||
      cudaMallocAsync(&Cg, M * N * sizeof(float2), st) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(TN_EHBM, "tn_contract_pair: unfused scratch allocation failed");
  }
  PermDesc pa{}, pb{}, pc{};
  pa.rank = d.nm + d.nk;  // A' row-major [m][k]
  for (int l = 0; l < d.nk; ++l) pa.st[l] = d.ak[l];
  for (int i = 0; i < d.nm; ++i) pa.st[d.nk + i] = d.am[i];
  pb.rank = d.nk + d.nn;  // B' row-major [k][n]
  for (int j = 0; j < d.nn; ++j) pb.st[j] = d.bn[j];
  for (int l = 0; l < d.nk; ++l) pb.st[d.nn + l] = d.bk[l];
  // C (its own layout) gathers from C' row-major [m][n]: bit p of C's index
  pc.rank = d.nm + d.nn;
  for (int i = 0; i < d.nm; ++i) pc.st[__builtin_ctz(d.cm[i])] = (int32_t)(N << i);
  for (int j = 0; j < d.nn; ++j) pc.st[__builtin_ctz(d.cn[j])] = int32_t(1) << j;
  cudaError_t e = launch_permute(A, Ap, pa, 1, 0, 0, st);
  if (e == cudaSuccess) e = launch_permute(B, Bp, pb, 1, 0, 0, st);
  if (e != cudaSuccess) { cleanup(); return fail(TN_ECUDA, "unfused permute: %s", cudaGetErrorString(e)); }
  int dev = 0;
  cudaGetDevice(&dev);
  cublasHandle_t h = cublas_handle(dev);
  if (!h) { cleanup(); return fail(TN_ECUDA, "cublasCreate failed"); }
  cublasSetStream(h, st);
  const cuComplex one = make_cuComplex(1.f, 0.f), zero = make_cuComplex(0.f, 0.f);
  // row-major C'[M][N] = A'[M][K] B'[K][N]  <=>  column-major C'^T = B'^T A'^T
  cublasStatus_t cs = cublasCgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)N, (int)M, (int)K, &one, (const cuComplex*)Bp,
                                  (int)N, (const cuComplex*)Ap, (int)K, &zero, (cuComplex*)Cg, (int)N);
  if (cs != CUBLAS_STATUS_SUCCESS) { cleanup(); return fail(TN_ECUDA, "cublasCgemm failed (%d)", (int)cs); }
  e = launch_permute(Cg, Cp, pc, 1, 0, 0, st);
  cleanup();
  if (e != cudaSuccess) return fail(TN_ECUDA, "unfused permute: %s", cudaGetErrorString(e));
  return TN_OK;
}

}  // namespace tn

using namespace tn;

// N <= 16 and K <= 16: the bandwidth kernel's shapes.
static bool d_is_vector(const std::vector<int>& la, const std::vector<int>& lb, const std::vector<int>& lc) {
  int nk = 0;
  for (int l : la)
    if (std::find(lb.begin(), lb.end(), l) != lb.end()) ++nk;
  const int nn = (int)lb.size() - nk;
  return (nn <= 4 && nk <= 4) || (nn <= 3 && nk <= 7) || (nn <= 8 && nk <= 2) || (nn == 5 && nk == 3);
}

extern "C" tn_status tn_set_wait_limit(int64_t polls) {
  const cudaError_t e = set_tc_wait_limit((long long)polls);
  if (e != cudaSuccess) return fail(TN_ECUDA, "tn_set_wait_limit: %s", cudaGetErrorString(e));
  return TN_OK;
}

extern "C" tn_status tn_contract_pair(const void* A, const int32_t* a_labels, int32_t ra, const void* B,
                                      const int32_t* b_labels, int32_t rb, void* Cv, const int32_t* c_labels,
                                      int32_t rc, int32_t precision, int32_t algo, void* stream) {
  if (!A || !B || !Cv) return fail(TN_EINVAL, "tn_contract_pair: NULL tensor");
  if (ra < 0 || rb < 0 || rc < 0 || ra > 30 || rb > 30 || rc > 30)
    return fail(TN_EINVAL, "tn_contract_pair: ranks must be in [0, 30]");
  if ((ra && !a_labels) || (rb && !b_labels) || (rc && !c_labels))
    return fail(TN_EINVAL, "tn_contract_pair: NULL labels");
  tn_status st = check_labels(a_labels, ra, b_labels, rb, c_labels, rc);
  if (st != TN_OK) return st;
  if (precision < TN_PREC_C64 || precision > TN_PREC_SCALED_BF16)
    return fail(TN_EINVAL, "tn_contract_pair: unknown precision %d", precision);
  return guarded("tn_contract_pair", [&]() -> tn_status {
  std::vector<int> la(a_labels, a_labels + ra), lb(b_labels, b_labels + rb), lc(c_labels, c_labels + rc);
  GemmDesc d;
  const bool vec_shape = d_is_vector(la, lb, lc);
  make_gemm_desc(la, lb, lc, d, vec_shape && (algo == TN_PAIR_AUTO || algo == TN_PAIR_VECTOR));
  d.units = 1;
  d.units_lo = 1;
  d.a_lo = d.a_hi = d.b_lo = d.b_hi = d.c_lo = d.c_hi = 0;
  cudaStream_t s = (cudaStream_t)stream;
  const float2* a = (const float2*)A;
  const float2* b = (const float2*)B;
  float2* c = (float2*)Cv;
  if (algo == TN_PAIR_AUTO) {
    if (vector_shape_ok(d)) algo = TN_PAIR_VECTOR;
    else if (reduce_shape_ok(d) && !(precision != TN_PREC_C64 && tc_shape_ok(d))) algo = TN_PAIR_REDUCE;
    else if (precision != TN_PREC_C64 && tc_shape_ok(d)) algo = TN_PAIR_FUSED_TC;
    else algo = TN_PAIR_FUSED_SIMT;
  }
  cudaError_t e;
  switch (algo) {
    case TN_PAIR_FUSED_SIMT: e = launch_gemm_simt(a, b, c, d, s); break;
    case TN_PAIR_VECTOR:
      if (!vector_shape_ok(d))
        return fail(TN_EINVAL, "tn_contract_pair: the vector kernel needs N, K <= 16, N <= 8 and K <= 128, N <= 256 "
                               "and K <= 4, or N = 32 and K = 8");
      e = launch_vector(a, b, c, d, s);
      break;
    case TN_PAIR_UNFUSED: return unfused(a, b, c, d, s);
    case TN_PAIR_REDUCE:
      if (!reduce_shape_ok(d))
        return fail(TN_EINVAL, "tn_contract_pair: the reduction kernel needs M N <= 64 and K >= 256");
      e = launch_reduce(a, b, c, d, s);
      break;
    case TN_PAIR_FUSED_TC:
    case TN_PAIR_GATHER_TC: {
      if (precision == TN_PREC_C64)
        return fail(TN_EINVAL, "tn_contract_pair: the tensor-core kernels need a 16-bit precision");
      if (algo == TN_PAIR_GATHER_TC && precision != TN_PREC_SPLIT_BF16)
        return fail(TN_EINVAL, "tn_contract_pair: the gathering tensor-core kernel runs split bf16 only");
      if (!tc_shape_ok(d)) return fail(TN_EINVAL, "tn_contract_pair: tensor-core kernels need M >= 128, N >= 16, K >= 8");
      std::lock_guard<std::mutex> lock(g_pair_mu);
      // operand planes, then 32 bytes for the scaled modes' maxima and exponents
      const size_t planes = algo == TN_PAIR_FUSED_TC ? (size_t)tc2_scratch_elems(d) * sizeof(uint16_t) : 0;
      PairDevState* ps = nullptr;
      tn_status pst = pair_state(planes + 32, ps);
      if (pst != TN_OK) return pst;
      int* err = ps->err;
      if (algo == TN_PAIR_FUSED_TC) {
        uint16_t* scratch = static_cast<uint16_t*>(ps->scratch);
        void* aux = static_cast<char*>(ps->scratch) + planes;
        switch (precision) {
          case TN_PREC_SPLIT_BF16: e = run_gemm_tc2(a, b, c, d, true, scratch, err, s); break;
          case TN_PREC_SPLIT_FP16: e = run_gemm_tc2_scaled(a, b, c, d, false, 4, scratch, aux, err, s); break;
          case TN_PREC_SCALED_FP16: e = run_gemm_tc2_scaled(a, b, c, d, false, 2, scratch, aux, err, s); break;
          default: e = run_gemm_tc2_scaled(a, b, c, d, true, 2, scratch, aux, err, s); break;
        }
      } else {
        e = launch_gemm_tc(a, b, c, d, true, 1.f, 1.f, err, s);
      }
      if (e == cudaSuccess) {
        int h = 0;
        cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && h) {
          const cudaError_t ce = cudaMemset(err, 0, sizeof(int));
          if (ce != cudaSuccess)
            return fail(TN_ECUDA, "tn_contract_pair: clearing the error word: %s", cudaGetErrorString(ce));
          return fail(TN_ETIMEOUT, "tn_contract_pair: a tensor-core pipeline wait expired (code %d)", h);
        }
      }
      break;
    }
    default: return fail(TN_EINVAL, "tn_contract_pair: algo %d not available for precision %d", algo, precision);
  }
  if (e != cudaSuccess) return fail(TN_ECUDA, "tn_contract_pair launch: %s", cudaGetErrorString(e));
  return TN_OK;
  });
}
