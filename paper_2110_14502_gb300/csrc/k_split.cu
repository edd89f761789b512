// Operand preparation for the TMA-fed tensor-core GEMM: gather a complex64
// operand through its per-bit strides (the index permutation) and write it
// once as four K-major 16-bit planes {re_hi, re_lo, im_hi, im_lo}, rows padded
// to the tile and K padded to the stage width with zeros.
//
// Paper: Sec. "Tensor Contraction Using Fused Permutation and Multiplication",
// imbalanced case (TTGT: one permuted copy of each operand feeds the GEMM; the
// position of every element comes from a pre-computed offset) and Sec. "A
// Mixed-Precision Computation Method via Adaptive Precision Scaling" (half
// precision operands: here each value is split as x = hi + lo,
// hi = rn16(x), lo = rn16(x - hi)).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "kernels.h"

namespace tn {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ uint16_t to16(float x, bool bf16) {
  return bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(x)) : __half_as_ushort(__float2half_rn(x));
}
__device__ __forceinline__ float from16(uint16_t h, bool bf16) {
  return bf16 ? __bfloat162float(__ushort_as_bfloat16(h)) : __half2float(__ushort_as_half(h));
}

// One thread: one row and one chunk of 8 K values -> one 16-byte store per plane.
__global__ void __launch_bounds__(NT) split_kernel(const float2* __restrict__ src, uint16_t* __restrict__ dst,
                                                   const SplitDesc d, bool bf16, float scale) {
  const int64_t rows = int64_t(1) << d.nrow;
  const int64_t K = int64_t(1) << d.nk;
  const int64_t kp = d.kp;
  const int64_t chunks = kp / 8;
  const int64_t z = blockIdx.y;
  src += (z % d.nlo) * d.lo + (z / d.nlo) * d.hi;
  const int64_t plane = (int64_t)d.rows_pad * kp;
  uint16_t* out = dst + z * 4 * plane;
  const int64_t total = (int64_t)d.rows_pad * chunks;
  for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < total; e += (int64_t)gridDim.x * NT) {
    const int64_t r = e / chunks, c = e % chunks;
    uint16_t rh[8], rl[8], ih[8], il[8];
    int32_t ro = 0;
    const bool rok = r < rows;
    if (rok)
      for (int i = 0; i < d.nrow; ++i)
        if ((r >> i) & 1) ro += d.row_st[i];
    float2 v[8];
    if (d.kvec && rok && c * 8 < K) {
      // 8 consecutive K values are contiguous: one 64-byte run
      int32_t ko = 0;
      const int64_t k0 = c * 8;
      for (int i = 3; i < d.nk; ++i)
        if ((k0 >> i) & 1) ko += d.k_st[i];
      const float4* p = reinterpret_cast<const float4*>(src + (int64_t)ro + ko);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 x = __ldg(p + q);
        v[2 * q] = make_float2(x.x, x.y);
        v[2 * q + 1] = make_float2(x.z, x.w);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t k = c * 8 + j;
        v[j] = make_float2(0.f, 0.f);
        if (rok && k < K) {
          int32_t ko = 0;
          for (int i = 0; i < d.nk; ++i)
            if ((k >> i) & 1) ko += d.k_st[i];
          v[j] = __ldg(src + (int64_t)ro + ko);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float re = v[j].x * scale, im = v[j].y * scale;
      rh[j] = to16(re, bf16);
      rl[j] = to16(re - from16(rh[j], bf16), bf16);
      ih[j] = to16(im, bf16);
      il[j] = to16(im - from16(ih[j], bf16), bf16);
    }
    const int64_t o = r * kp + c * 8;
    auto st16 = [&](uint16_t* p, const uint16_t* h) {
      uint4 w;
      w.x = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
      w.y = (uint32_t)h[2] | ((uint32_t)h[3] << 16);
      w.z = (uint32_t)h[4] | ((uint32_t)h[5] << 16);
      w.w = (uint32_t)h[6] | ((uint32_t)h[7] << 16);
      *reinterpret_cast<uint4*>(p) = w;
    };
    st16(out + o, rh);
    st16(out + plane + o, rl);
    st16(out + 2 * plane + o, ih);
    st16(out + 3 * plane + o, il);
  }
}

}  // namespace

cudaError_t launch_split(const float2* src, uint16_t* dst, const SplitDesc& d, int nz, bool bf16, float scale,
                         cudaStream_t s) {
  if (nz < 1 || nz > 65535 || d.kp % 8 != 0) return cudaErrorInvalidValue;
  const int64_t total = (int64_t)d.rows_pad * (d.kp / 8);
  const int64_t blocks = std::min<int64_t>((total + NT - 1) / NT, 152 * 8);
  split_kernel<<<dim3((unsigned)blocks, (unsigned)nz), NT, 0, s>>>(src, dst, d, bf16, scale);
  return cudaGetLastError();
}

namespace {
void split_desc(int nrow, const int32_t* row_st, int nk, const int32_t* k_st, int nlo, int64_t lo, int64_t hi,
                SplitDesc& sd) {
  sd.nrow = nrow;
  sd.nk = nk;
  sd.rows_pad = 1 << nrow;
  sd.kp = std::max(1 << nk, 32);
  sd.nlo = nlo;
  sd.lo = lo;
  sd.hi = hi;
  for (int i = 0; i < nrow; ++i) sd.row_st[i] = row_st[i];
  for (int i = 0; i < nk; ++i) sd.k_st[i] = k_st[i];
  // vector path: K >= 8 with its three lowest bits contiguous, 16-byte aligned rows
  bool rows_aligned = true;
  for (int i = 0; i < nrow; ++i) rows_aligned &= (row_st[i] % 2) == 0;
  sd.kvec = nk >= 3 && k_st[0] == 1 && k_st[1] == 2 && k_st[2] == 4 && rows_aligned && (lo % 2) == 0 && (hi % 2) == 0;
}
int distinct(const GemmDesc& d, int64_t lo, int64_t hi) {
  return (lo ? d.units_lo : 1) * (hi ? d.units / d.units_lo : 1);
}
}  // namespace

int64_t split_scratch_elems(const GemmDesc& d, bool which_b) {
  return which_b ? split_plane_elems(d.nn, d.nk) * distinct(d, d.b_lo, d.b_hi)
                 : split_plane_elems(d.nm, d.nk) * distinct(d, d.a_lo, d.a_hi);
}

int64_t tc2_scratch_elems(const GemmDesc& d) { return split_scratch_elems(d, false) + split_scratch_elems(d, true); }

cudaError_t split_operand(const float2* src, const GemmDesc& d, bool which_b, bool bf16, uint16_t* scratch,
                          PlaneOperand& out, cudaStream_t s) {
  const int64_t lo = which_b ? d.b_lo : d.a_lo, hi = which_b ? d.b_hi : d.a_hi;
  const int nrow = which_b ? d.nn : d.nm;
  SplitDesc sd;
  split_desc(nrow, which_b ? d.bn : d.am, d.nk, which_b ? d.bk : d.ak, lo ? d.units_lo : 1, lo, hi, sd);
  const int nz = distinct(d, lo, hi);
  cudaError_t e = launch_split(src, scratch, sd, nz, bf16, 1.f, s);
  const int64_t set = 4 * (int64_t(1) << nrow) * sd.kp * 2;
  out.base = scratch;
  out.kp = sd.kp;
  out.rows = int64_t(1) << nrow;
  out.nlo = lo ? d.units_lo : 1;
  out.nhi = hi ? d.units / d.units_lo : 1;
  out.st_lo = set;
  out.st_hi = set * out.nlo;
  return e;
}

bool planes_in_place(const float2* base, const GemmDesc& d, bool which_b, PlaneOperand& out) {
  const int nrow = which_b ? d.nn : d.nm;
  const int32_t* rs = which_b ? d.bn : d.am;
  const int32_t* ks = which_b ? d.bk : d.ak;
  const int64_t K = int64_t(1) << d.nk;
  if (K < 32) return false;
  for (int l = 0; l < d.nk; ++l)
    if (ks[l] != (int32_t(1) << l)) return false;
  for (int i = 0; i < nrow; ++i)
    if ((int64_t)rs[i] != (K << i)) return false;
  const int64_t lo = which_b ? d.b_lo : d.a_lo, hi = which_b ? d.b_hi : d.a_hi;
  out.base = reinterpret_cast<const uint16_t*>(base);
  out.kp = K;
  out.rows = int64_t(1) << nrow;
  out.nlo = lo ? d.units_lo : 1;
  out.nhi = hi ? d.units / d.units_lo : 1;
  out.st_lo = lo * 8;
  out.st_hi = hi * 8;
  return true;
}

cudaError_t run_gemm_tc2(const float2* A, const float2* B, float2* C, const GemmDesc& d, bool bf16, uint16_t* scratch,
                         int* err, cudaStream_t s) {
  PlaneOperand pa, pb;
  cudaError_t e = split_operand(A, d, false, bf16, scratch, pa, s);
  if (e != cudaSuccess) return e;
  e = split_operand(B, d, true, bf16, scratch + split_scratch_elems(d, false), pb, s);
  if (e != cudaSuccess) return e;
  return launch_gemm_tma(pa, pb, C, false, d, bf16, 1.f, err, s);
}

}  // namespace tn
