// Slice selection, cross-slice FP64 summation and a plain permutation kernel.
//
// Slice selection (paper: Sec. "A PEPS-based Simulation Method with an
// Optimized Slicing Strategy"): each (bitstring, slice) unit fixes the sliced
// indices to the bits of its slice id and the closed output indices to the
// bits of its bitstring; every leaf tensor carrying such an index contributes
// the corresponding sub-tensor.  Cross-slice sum (paper: Sec. "Scaling",
// global reduction of the slice results): the per-unit results are added in
// FP64 in unit order, so the sum order is fixed for a given call.
#include <algorithm>

#include "kernels.h"

namespace tn {

namespace {

__global__ void set_group_kernel(GroupInfo* slot, GroupInfo g) { *slot = g; }

__global__ void gather_kernel(const float2* __restrict__ store, float2* __restrict__ arena, int64_t arena_stride,
                              const LeafGather* __restrict__ descs, const GroupInfo* __restrict__ slot) {
  const GroupInfo g = *slot;
  const uint64_t* bits = g.bits;
  const LeafGather& L = descs[blockIdx.x];
  const int u = blockIdx.y;
  if (u >= g.units) return;
  const int64_t s = g.slice0 + u % g.nslice;
  const int64_t b = g.b0 + u / g.nslice;
  int64_t fixed_off = L.store_off;
  for (int f = 0; f < L.nfixed; ++f) {
    int src = L.fixed_src[f];
    int v;
    if (src >= 0) v = (int)((s >> src) & 1);
    else {
      int q = -src - 2;
      v = (int)((bits[b * g.words + (q >> 6)] >> (q & 63)) & 1);
    }
    if (v) fixed_off += L.fixed_stride[f];
  }
  const int sub = 1 << L.nkept;
  float2* dst = arena + (int64_t)u * arena_stride + L.dst_off;
  for (int e = threadIdx.x; e < sub; e += blockDim.x) {
    int64_t o = fixed_off;
    for (int p = 0; p < L.nkept; ++p)
      if ((e >> (L.nkept - 1 - p)) & 1) o += L.kept_stride[p];
    dst[e] = store[o];
  }
}

// The filter of the scaled precisions (Sec. "A Mixed-Precision Computation
// Method via Adaptive Precision Scaling": paths with under/overflow are kept
// out of the sum): a flagged unit adds nothing here and is listed for the
// host, which recomputes it in complex64 or counts it as discarded.
__global__ void accumulate_kernel(const float2* __restrict__ root, int64_t r_lo, int64_t r_hi,
                                  const int64_t* __restrict__ perm, int nperm, const GroupInfo* __restrict__ slot,
                                  const int* __restrict__ flag_s, const int* __restrict__ flag_u,
                                  int64_t* __restrict__ flagged, unsigned long long* __restrict__ nflagged,
                                  int cap) {
  const GroupInfo g = *slot;
  double2* acc = g.acc;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)g.nb * nperm) return;
  const int bl = (int)(idx / nperm);
  const int j = (int)(idx % nperm);
  double2 a = acc[(g.b0 + bl) * nperm + j];
  const float2* r = root + bl * r_hi + perm[j];
  for (int sl = 0; sl < g.nslice; ++sl) {
    if ((flag_s && flag_s[sl]) || (flag_u && flag_u[bl * g.nslice + sl])) {
      if (j == 0) {
        const unsigned long long k = atomicAdd(nflagged, 1ull);
        if ((int64_t)k < cap) flagged[k] = ((g.b0 + bl) << 32) | (g.slice0 + sl);
      }
      continue;
    }
    float2 v = r[sl * r_lo];
    a.x += (double)v.x;
    a.y += (double)v.y;
  }
  acc[(g.b0 + bl) * nperm + j] = a;
}

__global__ void permute_kernel(const float2* __restrict__ src, float2* __restrict__ dst, const PermDesc pd,
                               int64_t src_unit, int64_t dst_unit) {
  const int64_t n = int64_t(1) << pd.rank;
  const int64_t u = blockIdx.y;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = 0;
    for (int p = 0; p < pd.rank; ++p)
      if ((e >> p) & 1) o += pd.st[p];
    dst[u * dst_unit + e] = src[u * src_unit + o];
  }
}

}  // namespace

cudaError_t launch_set_group(GroupInfo* slot, const GroupInfo& g, cudaStream_t s) {
  set_group_kernel<<<1, 1, 0, s>>>(slot, g);
  return cudaGetLastError();
}

cudaError_t launch_gather(const float2* store, float2* arena, int64_t arena_stride, const LeafGather* descs,
                          int nleaves, const GroupInfo* slot, int units, cudaStream_t s) {
  if (nleaves == 0 || units == 0) return cudaSuccess;
  dim3 grid((unsigned)nleaves, (unsigned)units);
  gather_kernel<<<grid, 64, 0, s>>>(store, arena, arena_stride, descs, slot);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(const float2* root, int64_t r_lo, int64_t r_hi, const int64_t* perm, int nperm,
                              const GroupInfo* slot, int nb_max, const int* flag_s, const int* flag_u,
                              int64_t* flagged, unsigned long long* nflagged, int cap, cudaStream_t s) {
  const int64_t total = (int64_t)nb_max * nperm;
  const int nt = 256;
  accumulate_kernel<<<(unsigned)((total + nt - 1) / nt), nt, 0, s>>>(root, r_lo, r_hi, perm, nperm, slot, flag_s,
                                                                     flag_u, flagged, nflagged, cap);
  return cudaGetLastError();
}

cudaError_t launch_permute(const float2* src, float2* dst, const PermDesc& pd, int64_t units, int64_t src_unit,
                           int64_t dst_unit, cudaStream_t s) {
  int64_t n = int64_t(1) << pd.rank;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  permute_kernel<<<dim3(blocks, (unsigned)units), 256, 0, s>>>(src, dst, pd, src_unit, dst_unit);
  return cudaGetLastError();
}

}  // namespace tn
