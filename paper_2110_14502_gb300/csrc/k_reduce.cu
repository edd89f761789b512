// Bandwidth-bound contraction for steps with few outputs and a long
// contracted index: M N <= 64 outputs, K >= 256 (for example the last steps
// of a slice, which contract two wide tensors into the open-qubit batch).
//
// Paper: Sec. "Tensor Contraction Using Fused Permutation and
// Multiplication", imbalanced case: a memory-bound contraction whose operands
// are each streamed once.  Here one CTA takes one unit; thread t takes the
// contracted values k = t, t + 256, ..; it keeps partial sums of all M N
// outputs in registers, and the CTA combines them with warp shuffles and one
// pass through shared memory.  Consecutive threads read consecutive k, so the
// reads coalesce when the contracted indices are the operands' fastest ones
// (the planner's layout puts them there).
#include "kernels.h"

namespace tn {

namespace {

constexpr int NT = 256;
constexpr int LOW = 8;  // bits of k taken by the thread index

__device__ __forceinline__ int32_t bit_offset(int64_t x, int lo, int hi, const int32_t* st) {
  int32_t o = 0;
  for (int i = lo; i < hi; ++i)
    if ((x >> (i - lo)) & 1) o += st[i];
  return o;
}

template <int NM, int NN>
__global__ void __launch_bounds__(NT) reduce_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                                                    float2* __restrict__ C, const GemmDesc d) {
  constexpr int M = 1 << NM, N = 1 << NN;
  const int64_t ulo = blockIdx.x % d.units_lo, uhi = blockIdx.x / d.units_lo;
  A += ulo * d.a_lo + uhi * d.a_hi;
  B += ulo * d.b_lo + uhi * d.b_hi;
  C += ulo * d.c_lo + uhi * d.c_hi;
  __shared__ int32_t offA[M], offB[N];
  __shared__ float2 part[NT / 32][M * N];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < M) offA[tid] = bit_offset(tid, 0, NM, d.am);
  if (tid >= 64 && tid < 64 + N) offB[tid - 64] = bit_offset(tid - 64, 0, NN, d.bn);
  __syncthreads();
  float2 acc[M * N];
#pragma unroll
  for (int i = 0; i < M * N; ++i) acc[i] = make_float2(0.f, 0.f);
  const int32_t ka = bit_offset(tid, 0, LOW, d.ak), kb = bit_offset(tid, 0, LOW, d.bk);
  const int64_t nhigh = int64_t(1) << (d.nk - LOW);
  for (int64_t kh = 0; kh < nhigh; ++kh) {
    const int32_t oa = ka + bit_offset(kh, LOW, d.nk, d.ak), ob = kb + bit_offset(kh, LOW, d.nk, d.bk);
    float2 a[M], b[N];
#pragma unroll
    for (int m = 0; m < M; ++m) a[m] = __ldg(A + offA[m] + oa);
#pragma unroll
    for (int n = 0; n < N; ++n) b[n] = __ldg(B + offB[n] + ob);
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
      for (int n = 0; n < N; ++n) {
        float2& c = acc[m * N + n];
        c.x = fmaf(a[m].x, b[n].x, fmaf(-a[m].y, b[n].y, c.x));
        c.y = fmaf(a[m].x, b[n].y, fmaf(a[m].y, b[n].x, c.y));
      }
  }
#pragma unroll
  for (int i = 0; i < M * N; ++i) {
    float x = acc[i].x, y = acc[i].y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) part[warp][i] = make_float2(x, y);
  }
  __syncthreads();
  if (tid < M * N) {
    float2 s = part[0][tid];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) {
      s.x += part[w][tid].x;
      s.y += part[w][tid].y;
    }
    const int m = tid / N, n = tid % N;
    C[bit_offset(m, 0, NM, d.cm) + bit_offset(n, 0, NN, d.cn)] = s;
  }
}

template <int NM, int NN>
cudaError_t launch(const float2* A, const float2* B, float2* C, const GemmDesc& d, cudaStream_t s) {
  reduce_kernel<NM, NN><<<(unsigned)d.units, NT, 0, s>>>(A, B, C, d);
  return cudaGetLastError();
}

template <int NM>
cudaError_t launch_nn(const float2* A, const float2* B, float2* C, const GemmDesc& d, cudaStream_t s) {
  switch (d.nn) {
    case 0: return launch<NM, 0>(A, B, C, d, s);
    case 1: if constexpr (NM + 1 <= 6) return launch<NM, 1>(A, B, C, d, s); break;
    case 2: if constexpr (NM + 2 <= 6) return launch<NM, 2>(A, B, C, d, s); break;
    case 3: if constexpr (NM + 3 <= 6) return launch<NM, 3>(A, B, C, d, s); break;
    case 4: if constexpr (NM + 4 <= 6) return launch<NM, 4>(A, B, C, d, s); break;
    case 5: if constexpr (NM + 5 <= 6) return launch<NM, 5>(A, B, C, d, s); break;
    case 6: if constexpr (NM + 6 <= 6) return launch<NM, 6>(A, B, C, d, s); break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool reduce_shape_ok(const GemmDesc& d) { return d.nm + d.nn <= 6 && d.nk >= LOW && d.nk <= 30; }

cudaError_t launch_reduce(const float2* A, const float2* B, float2* C, const GemmDesc& d, cudaStream_t s) {
  if (!reduce_shape_ok(d) || d.units < 1 || d.units > (int64_t(1) << 31) - 1) return cudaErrorInvalidValue;
  switch (d.nm) {
    case 0: return launch_nn<0>(A, B, C, d, s);
    case 1: return launch_nn<1>(A, B, C, d, s);
    case 2: return launch_nn<2>(A, B, C, d, s);
    case 3: return launch_nn<3>(A, B, C, d, s);
    case 4: return launch_nn<4>(A, B, C, d, s);
    case 5: return launch_nn<5>(A, B, C, d, s);
    case 6: return launch_nn<6>(A, B, C, d, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tn
