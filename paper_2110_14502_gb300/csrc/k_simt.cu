// Fused permute-GEMM on FP32 CUDA cores (complex64 in, complex64 out).
//
// Paper: Sec. "Tensor Contraction Using Fused Permutation and Multiplication",
// dense case: the permutation of each operand is folded into the fetch of its
// tile rather than run as a separate pass.  Here every CTA computes the
// per-row / per-column element offsets of its tile from the operand's per-bit
// strides (the analogue of the paper's pre-computed position array), stages
// the permuted tiles in shared memory with the fetch order chosen for
// coalescing, and runs a complex FFMA micro-kernel (4 real FMAs per complex
// multiply-add, FP32 accumulation).
#include "kernels.h"

namespace tn {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ int32_t bit_offset(int64_t x, int nb, const int32_t* st) {
  int32_t o = 0;
  for (int i = 0; i < nb; ++i)
    if ((x >> i) & 1) o += st[i];
  return o;
}

__global__ void __launch_bounds__(NT) gemm_simt_kernel(const float2* __restrict__ A,
                                                        const float2* __restrict__ B,
                                                        float2* __restrict__ C, const GemmDesc d) {
  const int64_t M = int64_t(1) << d.nm, N = int64_t(1) << d.nn, K = int64_t(1) << d.nk;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int64_t ulo = blockIdx.z % d.units_lo, uhi = blockIdx.z / d.units_lo;
  A += ulo * d.a_lo + uhi * d.a_hi;
  B += ulo * d.b_lo + uhi * d.b_hi;
  C += ulo * d.c_lo + uhi * d.c_hi;
  __shared__ int32_t rowA[BM], rowC[BM], colB[BN], colC[BN], kA[BK], kB[BK];
  __shared__ float2 As[BK][BM], Bs[BK][BN];
  const int tid = threadIdx.x;
  if (tid < BM) {
    int64_t m = m0 + tid;
    rowA[tid] = m < M ? bit_offset(m, d.nm, d.am) : -1;
    rowC[tid] = m < M ? bit_offset(m, d.nm, d.cm) : -1;
  } else if (tid < BM + BN) {
    int64_t n = n0 + tid - BM;
    colB[tid - BM] = n < N ? bit_offset(n, d.nn, d.bn) : -1;
    colC[tid - BM] = n < N ? bit_offset(n, d.nn, d.cn) : -1;
  }
  const bool a_kfast = d.nk > 0 && d.ak[0] == 1;
  const bool b_kfast = d.nk > 0 && d.bk[0] == 1;
  const int ty = tid / 16, tx = tid % 16;
  float2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);

  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    if (tid < BK) {
      int64_t k = k0 + tid;
      kA[tid] = k < K ? bit_offset(k, d.nk, d.ak) : -1;
      kB[tid] = k < K ? bit_offset(k, d.nk, d.bk) : -1;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
      int e = tid + r * NT;
      int i = a_kfast ? e / BK : e % BM;
      int kk = a_kfast ? e % BK : e / BM;
      float2 v = make_float2(0.f, 0.f);
      if (rowA[i] >= 0 && kA[kk] >= 0) v = A[(int64_t)rowA[i] + kA[kk]];
      As[kk][i] = v;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
      int e = tid + r * NT;
      int j = b_kfast ? e / BK : e % BN;
      int kk = b_kfast ? e % BK : e / BN;
      float2 v = make_float2(0.f, 0.f);
      if (colB[j] >= 0 && kB[kk] >= 0) v = B[(int64_t)colB[j] + kB[kk]];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[r][c].x = fmaf(a[r].x, b[c].x, acc[r][c].x);
          acc[r][c].x = fmaf(-a[r].y, b[c].y, acc[r][c].x);
          acc[r][c].y = fmaf(a[r].x, b[c].y, acc[r][c].y);
          acc[r][c].y = fmaf(a[r].y, b[c].x, acc[r][c].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int i = ty * 4 + r;
    if (rowC[i] < 0) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int j = tx * 4 + c;
      if (colC[j] >= 0) C[(int64_t)rowC[i] + colC[j]] = acc[r][c];
    }
  }
}

}  // namespace

cudaError_t launch_gemm_simt(const float2* A, const float2* B, float2* C, const GemmDesc& d, cudaStream_t s) {
  int64_t M = int64_t(1) << d.nm, N = int64_t(1) << d.nn;
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)d.units);
  gemm_simt_kernel<<<grid, NT, 0, s>>>(A, B, C, d);
  return cudaGetLastError();
}

}  // namespace tn
