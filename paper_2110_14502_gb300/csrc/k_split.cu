// Operand preparation for the TMA-fed tensor-core GEMM: gather a complex64
// operand through its per-bit strides (the index permutation) and write it
// once as four K-major 16-bit planes {re_hi, re_lo, im_hi, im_lo} of K (>= 8)
// values per row; the GEMM's TMA box reads past a short K as zeros.
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

__device__ __forceinline__ int64_t src_offset_row(const SplitDesc& d, int64_t r) {
  int32_t ro = 0;
  for (int i = 0; i < d.nrow; ++i)
    if ((r >> i) & 1) ro += d.row_st[i];
  return ro;
}

// Load 8 consecutive K values (zero beyond K) of row r.
__device__ __forceinline__ void load8(const float2* __restrict__ src, const SplitDesc& d, bool rok, int64_t ro,
                                      int64_t c, float2* v) {
  const int64_t K = int64_t(1) << d.nk;
  if (d.kvec && rok && c * 8 < K) {
    // 8 consecutive K values are contiguous: one 64-byte run
    int32_t ko = 0;
    const int64_t k0 = c * 8;
    for (int i = 3; i < d.nk; ++i)
      if ((k0 >> i) & 1) ko += d.k_st[i];
    const float4* p = reinterpret_cast<const float4*>(src + ro + ko);
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
        v[j] = __ldg(src + ro + ko);
      }
    }
  }
}

// Largest |component| of each distinct tensor z (float bits, atomicMax).
__global__ void __launch_bounds__(NT) max_kernel(const float2* __restrict__ src, const SplitDesc d,
                                                 unsigned* __restrict__ maxbits) {
  const int64_t rows = int64_t(1) << d.nrow;
  const int64_t chunks = d.kp / 8;
  const int64_t z = blockIdx.y;
  src += (z % d.nlo) * d.lo + (z / d.nlo) * d.hi;
  float m = 0.f;
  const int64_t total = rows * chunks;
  for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < total; e += (int64_t)gridDim.x * NT) {
    const int64_t r = e / chunks, c = e % chunks;
    float2 v[8];
    load8(src, d, true, src_offset_row(d, r), c, v);
#pragma unroll
    for (int j = 0; j < 8; ++j) m = fmaxf(m, fmaxf(fabsf(v[j].x), fabsf(v[j].y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float wm[NT / 32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NT / 32; ++w) m = fmaxf(m, wm[w]);
    atomicMax(maxbits + z, __float_as_uint(m));
  }
}

// Exponent putting the maximum into [2^13, 2^14).
__device__ __forceinline__ int scale_exponent(float mx) {
  if (!(mx > 0.f) || !isfinite(mx)) return 0;
  int x;
  frexpf(mx, &x);  // mx in [2^(x-1), 2^x)
  return x - 14;
}

// One thread: one row and one chunk of 8 K values -> one 16-byte store per plane.
template <int NP>
__global__ void __launch_bounds__(NT) split_kernel(const float2* __restrict__ src, uint16_t* __restrict__ dst,
                                                   const SplitDesc d, bool bf16, const unsigned* __restrict__ maxbits,
                                                   int* __restrict__ e_out, float* __restrict__ m_out) {
  const int64_t rows = int64_t(1) << d.nrow;
  const int64_t kp = d.kp;
  const int64_t chunks = kp / 8;
  const int64_t z = blockIdx.y;
  src += (z % d.nlo) * d.lo + (z / d.nlo) * d.hi;
  int e = 0;
  if (maxbits) {
    const float mx = __uint_as_float(maxbits[z]);
    e = scale_exponent(mx);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      e_out[z] = e;
      m_out[z] = ldexpf(mx, -e);
    }
  }
  const int64_t plane = (int64_t)d.rows_pad * kp;
  uint16_t* out = dst + z * NP * plane;
  const int64_t total = (int64_t)d.rows_pad * chunks;
  for (int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x; q < total; q += (int64_t)gridDim.x * NT) {
    const int64_t r = q / chunks, c = q % chunks;
    const bool rok = r < rows;
    float2 v[8];
    load8(src, d, rok, rok ? src_offset_row(d, r) : 0, c, v);
    uint16_t h[NP][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float re = ldexpf(v[j].x, -e), im = ldexpf(v[j].y, -e);
      if (NP == 4) {
        h[0][j] = to16(re, bf16);
        h[1][j] = to16(re - from16(h[0][j], bf16), bf16);
        h[NP / 2][j] = to16(im, bf16);
        h[NP / 2 + 1][j] = to16(im - from16(h[NP / 2][j], bf16), bf16);
      } else {
        h[0][j] = to16(re, bf16);
        h[1][j] = to16(im, bf16);
      }
    }
    const int64_t o = r * kp + c * 8;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      uint4 w;
      w.x = (uint32_t)h[p][0] | ((uint32_t)h[p][1] << 16);
      w.y = (uint32_t)h[p][2] | ((uint32_t)h[p][3] << 16);
      w.z = (uint32_t)h[p][4] | ((uint32_t)h[p][5] << 16);
      w.w = (uint32_t)h[p][6] | ((uint32_t)h[p][7] << 16);
      *reinterpret_cast<uint4*>(out + p * plane + o) = w;
    }
  }
}

}  // namespace

cudaError_t launch_split(const float2* src, uint16_t* dst, const SplitDesc& d, int nz, bool bf16, int np,
                         unsigned* maxbits, int* e_out, float* m_out, cudaStream_t s, bool max_ready) {
  if (nz < 1 || nz > 65535 || d.kp % 8 != 0 || (np != 2 && np != 4)) return cudaErrorInvalidValue;
  const int64_t total = (int64_t)d.rows_pad * (d.kp / 8);
  const int64_t blocks = std::min<int64_t>((total + NT - 1) / NT, 152 * 8);
  if (maxbits && !max_ready) {
    max_kernel<<<dim3((unsigned)blocks, (unsigned)nz), NT, 0, s>>>(src, d, maxbits);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (np == 4)
    split_kernel<4><<<dim3((unsigned)blocks, (unsigned)nz), NT, 0, s>>>(src, dst, d, bf16, maxbits, e_out, m_out);
  else
    split_kernel<2><<<dim3((unsigned)blocks, (unsigned)nz), NT, 0, s>>>(src, dst, d, bf16, maxbits, e_out, m_out);
  return cudaGetLastError();
}

namespace {
void split_desc(int nrow, const int32_t* row_st, int nk, const int32_t* k_st, int nlo, int64_t lo, int64_t hi,
                SplitDesc& sd) {
  sd.nrow = nrow;
  sd.nk = nk;
  sd.rows_pad = 1 << nrow;
  sd.kp = 1 << nk;  // tensor-core shapes have K >= 8: whole 16-byte chunks, no padding
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

int64_t split_scratch_elems(const GemmDesc& d, bool which_b, int np) {
  return which_b ? split_plane_elems(d.nn, d.nk, np) * distinct(d, d.b_lo, d.b_hi)
                 : split_plane_elems(d.nm, d.nk, np) * distinct(d, d.a_lo, d.a_hi);
}

int64_t tc2_scratch_elems(const GemmDesc& d) { return split_scratch_elems(d, false, 4) + split_scratch_elems(d, true, 4); }

cudaError_t split_operand(const float2* src, const GemmDesc& d, bool which_b, bool bf16, int np, bool scaled,
                          unsigned* maxbits, int* e_out, float* m_out, uint16_t* scratch, PlaneOperand& out,
                          cudaStream_t s, bool max_ready) {
  const int64_t lo = which_b ? d.b_lo : d.a_lo, hi = which_b ? d.b_hi : d.a_hi;
  const int nrow = which_b ? d.nn : d.nm;
  SplitDesc sd;
  split_desc(nrow, which_b ? d.bn : d.am, d.nk, which_b ? d.bk : d.ak, lo ? d.units_lo : 1, lo, hi, sd);
  const int nz = distinct(d, lo, hi);
  cudaError_t e = launch_split(src, scratch, sd, nz, bf16, np, scaled ? maxbits : nullptr, e_out, m_out, s, max_ready);
  const int64_t set = (int64_t)np * (int64_t(1) << nrow) * sd.kp * 2;
  out.base = scratch;
  out.np = np;
  out.kp = sd.kp;
  out.rows = int64_t(1) << nrow;
  out.nlo = lo ? d.units_lo : 1;
  out.nhi = hi ? d.units / d.units_lo : 1;
  out.st_lo = set;
  out.st_hi = set * out.nlo;
  return e;
}

bool planes_in_place(const float2* base, const GemmDesc& d, bool which_b, int np, PlaneOperand& out) {
  const int nrow = which_b ? d.nn : d.nm;
  const int32_t* rs = which_b ? d.bn : d.am;
  const int32_t* ks = which_b ? d.bk : d.ak;
  const int64_t K = int64_t(1) << d.nk;
  if (K < 8) return false;
  for (int l = 0; l < d.nk; ++l)
    if (ks[l] != (int32_t(1) << l)) return false;
  for (int i = 0; i < nrow; ++i)
    if ((int64_t)rs[i] != (K << i)) return false;
  const int64_t lo = which_b ? d.b_lo : d.a_lo, hi = which_b ? d.b_hi : d.a_hi;
  out.base = reinterpret_cast<const uint16_t*>(base);
  out.np = np;
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
  cudaError_t e = split_operand(A, d, false, bf16, 4, false, nullptr, nullptr, nullptr, scratch, pa, s);
  if (e != cudaSuccess) return e;
  e = split_operand(B, d, true, bf16, 4, false, nullptr, nullptr, nullptr, scratch + split_scratch_elems(d, false, 4),
                    pb, s);
  if (e != cudaSuccess) return e;
  const ScaleIO none{};
  return launch_gemm_tma(pa, pb, C, false, d, bf16, none, err, s);
}

cudaError_t run_gemm_tc2_scaled(const float2* A, const float2* B, float2* C, const GemmDesc& d, bool bf16, int np,
                                uint16_t* scratch, void* aux, int* err, cudaStream_t s) {
  unsigned* mx = reinterpret_cast<unsigned*>(aux);
  int* ex = reinterpret_cast<int*>(mx + 2);
  float* ms = reinterpret_cast<float*>(ex + 2);
  cudaError_t e = cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned), s);
  PlaneOperand pa, pb;
  if (e == cudaSuccess) e = split_operand(A, d, false, bf16, np, true, mx, ex, ms, scratch, pa, s);
  if (e == cudaSuccess)
    e = split_operand(B, d, true, bf16, np, true, mx + 1, ex + 1, ms + 1,
                      scratch + split_scratch_elems(d, false, np), pb, s);
  if (e != cudaSuccess) return e;
  ScaleIO sio{};
  sio.ea = ex;
  sio.ma = ms;
  sio.eb = ex + 1;
  sio.mb = ms + 1;
  return launch_gemm_tma(pa, pb, C, false, d, bf16, sio, err, s);
}

}  // namespace tn
