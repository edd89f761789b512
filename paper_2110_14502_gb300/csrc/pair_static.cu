// tn_contract_pair_noalloc: the tensor-core pairwise contraction without any
// device allocation.
//
// Why it exists: the regular tensor-core path of tn_contract_pair takes its
// scratch memory (the split 16-bit operand planes) from cudaMalloc, growing a
// per-device buffer whenever a call needs more.  Some callers cannot let a
// library allocate:
//   - a host framework whose caching allocator already holds nearly all free
//     device memory (PyTorch reserves HBM in large blocks), so a cudaMalloc
//     from the library fails although the framework could have served it;
//   - serving loops with a fixed memory budget or strict latency targets, where
//     an allocator call (and the synchronisation cudaMalloc may imply) is not
//     allowed on the request path;
//   - code that must not touch the allocator while another thread is
//     capturing work into a CUDA graph.
// This entry point takes its scratch from one file-scope device array of a
// fixed size instead.
//
// Behaviour:
//   - Scratch limit: kStaticScratchElems 16-bit values (64 MiB).  A call whose
//     split operand planes need more is rejected with TN_EINVAL before any work
//     is queued.  Every GPU that loads the library keeps this array (and a
//     4-byte error word) until the process exits.
//   - Set-up: the first call on a device (with that device current) looks up
//     the device address of the array and of the error word with
//     cudaGetSymbolAddress and clears the error word; make that first call
//     before any stream capture.  Later calls only reuse the cached addresses.
//   - Sharing: every call on a device uses the same array, and the array keeps
//     the last call's contents.  The split pass overwrites every value the GEMM
//     reads (zero padding included), so nothing has to be cleared between
//     calls; but two calls whose work overlaps on the GPU (different streams,
//     or different host threads) race on the array and give wrong results:
//     serialise them.
//   - The call allocates nothing: no cudaMalloc, cudaFree, cudaMallocAsync or
//     allocating library routine.  It clears the shared error word on
//     `stream` before its launch and reads it back afterwards, so it returns
//     once the contraction has finished on `stream`, and a wait that expired
//     in an earlier call is never reported again.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.h"
#include "tn_internal.h"

namespace tn {

constexpr int64_t kStaticScratchElems = int64_t(1) << 25;  // 2^25 x 2 bytes = 64 MiB

static __device__ __align__(256) uint16_t g_static_scratch[kStaticScratchElems];
static __device__ int g_static_err;

namespace {

struct DevSlots {
  uint16_t* scratch = nullptr;
  int* err = nullptr;
  bool ready = false;
};

std::mutex g_mu;
std::vector<DevSlots> g_slots;

// Same rules as tn_contract_pair: each output label in exactly one operand,
// every operand label contracted or kept, no label repeated within a tensor.
tn_status check_labels(const int32_t* la, int ra, const int32_t* lb, int rb, const int32_t* lc, int rc) {
  auto has = [](const int32_t* l, int r, int x) { return std::find(l, l + r, x) != l + r; };
  auto distinct = [](const int32_t* l, int r) {
    std::vector<int> v(l, l + r);
    std::sort(v.begin(), v.end());
    return std::adjacent_find(v.begin(), v.end()) == v.end();
  };
  if (!distinct(la, ra) || !distinct(lb, rb) || !distinct(lc, rc))
    return fail(TN_EINVAL, "tn_contract_pair_noalloc: repeated label within a tensor");
  for (int i = 0; i < rc; ++i)
    if (has(la, ra, lc[i]) == has(lb, rb, lc[i]))
      return fail(TN_EINVAL, "tn_contract_pair_noalloc: output label %d must appear in exactly one operand", lc[i]);
  for (int i = 0; i < ra; ++i)
    if (!has(lb, rb, la[i]) && !has(lc, rc, la[i]))
      return fail(TN_EINVAL, "tn_contract_pair_noalloc: label %d of A is neither contracted nor in C", la[i]);
  for (int i = 0; i < rb; ++i)
    if (!has(la, ra, lb[i]) && !has(lc, rc, lb[i]))
      return fail(TN_EINVAL, "tn_contract_pair_noalloc: label %d of B is neither contracted nor in C", lb[i]);
  return TN_OK;
}

// Per-device set-up: device addresses of the scratch array and error word.
tn_status static_slots(DevSlots& out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(TN_ECUDA, "tn_contract_pair_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
  std::lock_guard<std::mutex> g(g_mu);
  if ((int)g_slots.size() <= dev) g_slots.resize(dev + 1);
  DevSlots& s = g_slots[dev];
  if (!s.ready) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess)
      return fail(TN_ECUDA, "tn_contract_pair_noalloc: cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    s.scratch = (uint16_t*)p;
    e = cudaGetSymbolAddress(&p, g_static_err);
    if (e != cudaSuccess)
      return fail(TN_ECUDA, "tn_contract_pair_noalloc: cudaGetSymbolAddress(err): %s", cudaGetErrorString(e));
    s.err = (int*)p;
    e = cudaMemset(s.err, 0, sizeof(int));
    if (e != cudaSuccess) return fail(TN_ECUDA, "tn_contract_pair_noalloc: clearing the error word: %s", cudaGetErrorString(e));
    s.ready = true;
  }
  out = s;
  return TN_OK;
}

}  // namespace

}  // namespace tn

using namespace tn;

extern "C" tn_status tn_contract_pair_noalloc(const void* A, const int32_t* a_labels, int32_t ra, const void* B,
                                              const int32_t* b_labels, int32_t rb, void* Cv,
                                              const int32_t* c_labels, int32_t rc, void* stream) {
  if (!A || !B || !Cv) return fail(TN_EINVAL, "tn_contract_pair_noalloc: NULL tensor");
  if (ra < 0 || rb < 0 || rc < 0 || ra > 30 || rb > 30 || rc > 30)
    return fail(TN_EINVAL, "tn_contract_pair_noalloc: ranks must be in [0, 30]");
  if ((ra && !a_labels) || (rb && !b_labels) || (rc && !c_labels))
    return fail(TN_EINVAL, "tn_contract_pair_noalloc: NULL labels");
  tn_status st = check_labels(a_labels, ra, b_labels, rb, c_labels, rc);
  if (st != TN_OK) return st;
  return guarded("tn_contract_pair_noalloc", [&]() -> tn_status {
  std::vector<int> la(a_labels, a_labels + ra), lb(b_labels, b_labels + rb), lc(c_labels, c_labels + rc);
  GemmDesc d;
  make_gemm_desc(la, lb, lc, d);
  if (!tc_shape_ok(d))
    return fail(TN_EINVAL, "tn_contract_pair_noalloc: needs M >= 128, N >= 16, K >= 8 (got 2^%d, 2^%d, 2^%d)", d.nm,
                d.nn, d.nk);
  const int64_t need = tc2_scratch_elems(d);
  if (need > kStaticScratchElems)
    return fail(TN_EINVAL,
                "tn_contract_pair_noalloc: the split operands need %lld bytes of scratch; the static buffer holds "
                "%lld bytes",
                (long long)(need * 2), (long long)(kStaticScratchElems * 2));
  DevSlots slots;
  st = static_slots(slots);
  if (st != TN_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // this call's error word starts at zero, in stream order before its kernels
  cudaError_t e = cudaMemsetAsync(slots.err, 0, sizeof(int), s);
  if (e != cudaSuccess)
    return fail(TN_ECUDA, "tn_contract_pair_noalloc: clearing the error word: %s", cudaGetErrorString(e));
  e = run_gemm_tc2((const float2*)A, (const float2*)B, (float2*)Cv, d, true, slots.scratch, slots.err, s);
  if (e != cudaSuccess) return fail(TN_ECUDA, "tn_contract_pair_noalloc launch: %s", cudaGetErrorString(e));
  int h = 0;
  e = cudaMemcpyAsync(&h, slots.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(TN_ECUDA, "tn_contract_pair_noalloc: %s", cudaGetErrorString(e));
  if (h) return fail(TN_ETIMEOUT, "tn_contract_pair_noalloc: a tensor-core pipeline wait expired (code %d)", h);
  return TN_OK;
  });
}
