// Bandwidth-bound contraction for vector-like steps (N <= 16 and K <= 16,
// N <= 8 and K <= 128, N <= 256 and K <= 4, or N = 32 and K = 8).  The output
// is complex64, or a tensor-core consumer's four 16-bit split planes.
//
// Paper: Sec. "Tensor Contraction Using Fused Permutation and
// Multiplication", imbalanced case (a high-rank tensor against a rank-4 one):
// the small operand is kept in fast memory and the large one is streamed once.
// Here the small operand B (K x N complex) sits in shared memory, each thread
// owns rows m of the large operand, reads its K elements and writes its N
// outputs; consecutive threads take consecutive m, so with the step's bit
// order (bit 0 = most contiguous index) both the stream of A and the store of
// C coalesce.  The row offsets come from two 32-entry position tables per
// CTA plus one CTA base (the bits of m are disjoint, so offsets add).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "kernels.h"

namespace tn {

namespace {

constexpr int NT = 256;
constexpr int PER = 4;                 // rows per thread
constexpr int CH_BITS = 10;            // 1024 rows per CTA
constexpr int CH = 1 << CH_BITS;
static_assert(NT * PER == CH, "chunk");

__device__ __forceinline__ int32_t bit_offset(int64_t x, int nb, const int32_t* st) {
  int32_t o = 0;
  for (int i = 0; i < nb; ++i)
    if ((x >> i) & 1) o += st[i];
  return o;
}

__device__ __forceinline__ float cmax(float m, float2 v) { return fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y))); }

// acc[n] += a0 B[k][n] + a1 B[k+1][n] for every n (rows Bk0, Bk1 of B in
// shared memory), B read two columns per 16-byte load.
__device__ __forceinline__ void cmac2(float2& c, float2 a0, float2 a1, float2 b0, float2 b1) {
  c.x = fmaf(a0.x, b0.x, fmaf(-a0.y, b0.y, c.x));
  c.y = fmaf(a0.x, b0.y, fmaf(a0.y, b0.x, c.y));
  c.x = fmaf(a1.x, b1.x, fmaf(-a1.y, b1.y, c.x));
  c.y = fmaf(a1.x, b1.y, fmaf(a1.y, b1.x, c.y));
}
template <int N>
__device__ __forceinline__ void mac_pair(float2 (&acc)[N], const float2* Bk0, const float2* Bk1, float2 a0, float2 a1) {
  if constexpr (N >= 2) {
#pragma unroll
    for (int n = 0; n < N; n += 2) {
      const float4 p0 = *reinterpret_cast<const float4*>(Bk0 + n), p1 = *reinterpret_cast<const float4*>(Bk1 + n);
      cmac2(acc[n], a0, a1, make_float2(p0.x, p0.y), make_float2(p1.x, p1.y));
      cmac2(acc[n + 1], a0, a1, make_float2(p0.z, p0.w), make_float2(p1.z, p1.w));
    }
  } else {
    cmac2(acc[0], a0, a1, Bk0[0], Bk1[0]);
  }
}

// The largest |component| this warp wrote, into the launch unit's slot (a
// scaled split of the output then needs no pass of its own for it).
__device__ __forceinline__ void record_max(unsigned* maxbits, float m) {
  if (!maxbits) return;
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxbits + blockIdx.y, __float_as_uint(m));
}

__device__ __forceinline__ uint16_t h16(float x, int bf16) {
  return bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(x)) : __half_as_ushort(__float2half_rn(x));
}
__device__ __forceinline__ float f16(uint16_t h, int bf16) {
  return bf16 ? __bfloat162float(__ushort_as_bfloat16(h)) : __half2float(__ushort_as_half(h));
}

// One output value: complex64 (mode 0), or the four 16-bit planes re_hi,
// re_lo, im_hi, im_lo (mode 2; hi = rn16(x), lo = rn16(x - hi), the split
// pass's roundings) at the same element offset.
__device__ __forceinline__ void emit(const VecOut& o, float2* C, int64_t off, float2 v, float& mx) {
  mx = cmax(mx, v);
  if (o.mode == 0) {
    C[off] = v;
  } else {
    uint16_t* P = reinterpret_cast<uint16_t*>(C);
    const float re = v.x, im = v.y;
    const uint16_t rh = h16(re, o.bf16), ih = h16(im, o.bf16);
    P[off] = rh;
    P[o.plane + off] = h16(re - f16(rh, o.bf16), o.bf16);
    P[2 * o.plane + off] = ih;
    P[3 * o.plane + off] = h16(im - f16(ih, o.bf16), o.bf16);
  }
}

template <int NK, int NN>
__global__ void __launch_bounds__(NT) vector_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                                                    float2* __restrict__ C, const GemmDesc d,
                                                    const VecOut o) {
  constexpr int K = 1 << NK, N = 1 << NN;
  const int64_t M = int64_t(1) << d.nm;
  const int64_t ulo = blockIdx.y % d.units_lo, uhi = blockIdx.y / d.units_lo;
  A += ulo * d.a_lo + uhi * d.a_hi;
  B += ulo * d.b_lo + uhi * d.b_hi;
  C += ulo * d.c_lo + uhi * d.c_hi;
  __shared__ float2 Bs[K * N];
  __shared__ int32_t kA[K], nC[N];
  __shared__ int32_t tAlo[32], tAhi[32], tClo[32], tChi[32];
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * CH;
  for (int e = tid; e < K * N; e += NT) {
    int k = e / N, n = e % N;
    Bs[e] = B[bit_offset(k, NK, d.bk) + bit_offset(n, NN, d.bn)];
  }
  if (tid < K) kA[tid] = bit_offset(tid, NK, d.ak);
  if (tid >= 64 && tid < 64 + N) nC[tid - 64] = bit_offset(tid - 64, NN, d.cn);
  const int lb = d.nm < CH_BITS ? d.nm : CH_BITS;  // bits of m inside the chunk
  if (tid >= 128 && tid < 160) {
    int x = tid - 128;
    int b0 = lb < 5 ? lb : 5;
    tAlo[x] = x < (1 << b0) ? bit_offset(x, b0, d.am) : 0;
    tClo[x] = x < (1 << b0) ? bit_offset(x, b0, d.cm) : 0;
  }
  if (tid >= 160 && tid < 192) {
    int x = tid - 160;
    int b1 = lb > 5 ? lb - 5 : 0;
    tAhi[x] = x < (1 << b1) ? bit_offset(x, b1, d.am + 5) : 0;
    tChi[x] = x < (1 << b1) ? bit_offset(x, b1, d.cm + 5) : 0;
  }
  // CTA base offsets from the bits of m above the chunk
  __shared__ int32_t baseA, baseC;
  if (tid == 0) {
    int32_t oa = 0, oc = 0;
    for (int i = CH_BITS; i < d.nm; ++i)
      if ((base >> i) & 1) { oa += d.am[i]; oc += d.cm[i]; }
    baseA = oa;
    baseC = oc;
  }
  __syncthreads();
  float mx = 0.f;
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    int loc = tid + r * NT;
    if (base + loc >= M) break;
    int32_t oa = baseA + tAlo[loc & 31] + tAhi[loc >> 5];
    int32_t oc = baseC + tClo[loc & 31] + tChi[loc >> 5];
    float2 a[K];
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = __ldg(A + (int64_t)oa + kA[k]);
#pragma unroll
    for (int n = 0; n < N; ++n) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float2 b = Bs[k * N + n];
        acc.x = fmaf(a[k].x, b.x, acc.x);
        acc.x = fmaf(-a[k].y, b.y, acc.x);
        acc.y = fmaf(a[k].x, b.y, acc.y);
        acc.y = fmaf(a[k].y, b.x, acc.y);
      }
      emit(o, C, (int64_t)oc + nC[n], acc, mx);
    }
  }
  record_max(o.maxbits, mx);
}

// Wide B with a very short contracted index (K <= 4, N = 32..256): the
// outer-product-like steps that expand a tensor.  The row's K values stay in
// registers while the thread walks the N columns, so the registers do not grow
// with N; B (K N <= 1024 complex) sits in shared memory.
template <int NK, int NN>
__global__ void __launch_bounds__(NT) vector_wide_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                                                         float2* __restrict__ C, const GemmDesc d,
                                                         const VecOut o, int pair_k) {
  constexpr int K = 1 << NK, N = 1 << NN;
  static_assert(K * N <= 1024, "B must fit in shared memory");
  const int64_t M = int64_t(1) << d.nm;
  const int64_t ulo = blockIdx.y % d.units_lo, uhi = blockIdx.y / d.units_lo;
  A += ulo * d.a_lo + uhi * d.a_hi;
  B += ulo * d.b_lo + uhi * d.b_hi;
  C += ulo * d.c_lo + uhi * d.c_hi;
  __shared__ float2 Bs[K * N];
  __shared__ int32_t kA[K], nC[N];
  __shared__ int32_t tAlo[32], tAhi[32], tClo[32], tChi[32];
  __shared__ int32_t baseA, baseC;
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * CH;
  for (int e = tid; e < K * N; e += NT) {
    const int k = e / N, n = e % N;
    Bs[e] = B[bit_offset(k, NK, d.bk) + bit_offset(n, NN, d.bn)];
  }
  if (tid < K) kA[tid] = bit_offset(tid, NK, d.ak);
  for (int n = tid; n < N; n += NT) nC[n] = bit_offset(n, NN, d.cn);
  const int lb = d.nm < CH_BITS ? d.nm : CH_BITS;
  if (tid >= 128 && tid < 160) {
    const int x = tid - 128, b0 = lb < 5 ? lb : 5;
    tAlo[x] = x < (1 << b0) ? bit_offset(x, b0, d.am) : 0;
    tClo[x] = x < (1 << b0) ? bit_offset(x, b0, d.cm) : 0;
  }
  if (tid >= 160 && tid < 192) {
    const int x = tid - 160, b1 = lb > 5 ? lb - 5 : 0;
    tAhi[x] = x < (1 << b1) ? bit_offset(x, b1, d.am + 5) : 0;
    tChi[x] = x < (1 << b1) ? bit_offset(x, b1, d.cm + 5) : 0;
  }
  if (tid == 192) {
    int32_t oa = 0, oc = 0;
    for (int i = CH_BITS; i < d.nm; ++i)
      if ((base >> i) & 1) { oa += d.am[i]; oc += d.cm[i]; }
    baseA = oa;
    baseC = oc;
  }
  __syncthreads();
  float mx = 0.f;
#pragma unroll 1
  for (int r = 0; r < PER; ++r) {
    const int loc = tid + r * NT;
    if (base + loc >= M) break;
    const int32_t oa = baseA + tAlo[loc & 31] + tAhi[loc >> 5];
    const int32_t oc = baseC + tClo[loc & 31] + tChi[loc >> 5];
    float2 a[K];
    if (K >= 2 && pair_k) {
#pragma unroll
      for (int k = 0; k < K; k += 2) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(A + (int64_t)oa + kA[k]));
        a[k] = make_float2(x.x, x.y);
        a[k + 1 < K ? k + 1 : k] = make_float2(x.z, x.w);
      }
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) a[k] = __ldg(A + (int64_t)oa + kA[k]);
    }
#pragma unroll 8
    for (int n = 0; n < N; ++n) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float2 b = Bs[k * N + n];
        acc.x = fmaf(a[k].x, b.x, acc.x);
        acc.x = fmaf(-a[k].y, b.y, acc.x);
        acc.y = fmaf(a[k].x, b.y, acc.y);
        acc.y = fmaf(a[k].y, b.x, acc.y);
      }
      emit(o, C, (int64_t)oc + nC[n], acc, mx);
    }
  }
  record_max(o.maxbits, mx);
}

// Longer contracted index (K = 32..128) with a narrow B (N <= 8, N K <= 1024):
// the same streaming layout, but each row's K values are consumed into N
// running sums instead of being held in registers.  With pair_k (K bit 0 of A
// has stride 1 and every pair starts on a 16-byte boundary) a row's K values
// arrive two per 16-byte load.
template <int NK, int NN>
__global__ void __launch_bounds__(NT) vector_long_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                                                         float2* __restrict__ C, const GemmDesc d, int pair_k,
                                                         const VecOut o) {
  constexpr int K = 1 << NK, N = 1 << NN;
  static_assert(K * N <= 1024, "B must fit in shared memory");
  const int64_t M = int64_t(1) << d.nm;
  const int64_t ulo = blockIdx.y % d.units_lo, uhi = blockIdx.y / d.units_lo;
  A += ulo * d.a_lo + uhi * d.a_hi;
  B += ulo * d.b_lo + uhi * d.b_hi;
  C += ulo * d.c_lo + uhi * d.c_hi;
  __shared__ __align__(16) float2 Bs[K * N];
  __shared__ int32_t kA[K], nC[N];
  __shared__ int32_t tAlo[32], tAhi[32], tClo[32], tChi[32];
  __shared__ int32_t baseA, baseC;
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * CH;
  for (int e = tid; e < K * N; e += NT) {
    const int k = e / N, n = e % N;
    Bs[e] = B[bit_offset(k, NK, d.bk) + bit_offset(n, NN, d.bn)];
  }
  for (int k = tid; k < K; k += NT) kA[k] = bit_offset(k, NK, d.ak);
  if (tid >= 192 && tid < 192 + N) nC[tid - 192] = bit_offset(tid - 192, NN, d.cn);
  const int lb = d.nm < CH_BITS ? d.nm : CH_BITS;
  if (tid >= 128 && tid < 160) {
    const int x = tid - 128, b0 = lb < 5 ? lb : 5;
    tAlo[x] = x < (1 << b0) ? bit_offset(x, b0, d.am) : 0;
    tClo[x] = x < (1 << b0) ? bit_offset(x, b0, d.cm) : 0;
  }
  if (tid >= 160 && tid < 192) {
    const int x = tid - 160, b1 = lb > 5 ? lb - 5 : 0;
    tAhi[x] = x < (1 << b1) ? bit_offset(x, b1, d.am + 5) : 0;
    tChi[x] = x < (1 << b1) ? bit_offset(x, b1, d.cm + 5) : 0;
  }
  if (tid == 0) {
    int32_t oa = 0, oc = 0;
    for (int i = CH_BITS; i < d.nm; ++i)
      if ((base >> i) & 1) { oa += d.am[i]; oc += d.cm[i]; }
    baseA = oa;
    baseC = oc;
  }
  __syncthreads();
  float mx = 0.f;
#pragma unroll 1
  for (int r = 0; r < PER; ++r) {
    const int loc = tid + r * NT;
    if (base + loc >= M) break;
    const int32_t oa = baseA + tAlo[loc & 31] + tAhi[loc >> 5];
    const int32_t oc = baseC + tClo[loc & 31] + tChi[loc >> 5];
    float2 acc[N];
#pragma unroll
    for (int n = 0; n < N; ++n) acc[n] = make_float2(0.f, 0.f);
    if (pair_k) {
#pragma unroll 4
      for (int k = 0; k < K; k += 2) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(A + (int64_t)oa + kA[k]));
        mac_pair<N>(acc, Bs + k * N, Bs + (k + 1) * N, make_float2(x.x, x.y), make_float2(x.z, x.w));
      }
    } else {
#pragma unroll 8
      for (int k = 0; k < K; ++k) {
        const float2 a = __ldg(A + (int64_t)oa + kA[k]);
#pragma unroll
        for (int n = 0; n < N; ++n) {
          const float2 b = Bs[k * N + n];
          acc[n].x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc[n].x));
          acc[n].y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc[n].y));
        }
      }
    }
#pragma unroll
    for (int n = 0; n < N; ++n) {
      emit(o, C, (int64_t)oc + nC[n], acc[n], mx);
    }
  }
  record_max(o.maxbits, mx);
}

// Rows whose K values are contiguous (A's K bit i has stride 2^i, K >= 8):
// a warp copies 32 rows' next KC = min(K, 16) values into shared memory with
// 16-byte cp.async (every load instruction reads whole 128-byte lines, where a
// thread-per-row load touches 32 lines a few bytes at a time), double-buffered
// per warp, and each lane then runs its own row from shared memory into N
// running sums.  Row pitch KC + 2 complex keeps the lanes' 16-byte reads of a
// quarter-warp on distinct banks.  A CTA of SW warps owns 1024 consecutive
// rows (M >= 32: every warp group of 32 rows is full).
constexpr int SW = 4;
constexpr int SNT = SW * 32;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <int NK, int NN>
__global__ void __launch_bounds__(SNT) vector_staged_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                                                            float2* __restrict__ C, const GemmDesc d,
                                                            const VecOut o) {
  constexpr int K = 1 << NK, N = 1 << NN;
  constexpr int KC = K < 16 ? K : 16;    // K values per stage
  constexpr int PITCH = KC + 2;          // complex per staged row
  constexpr int LPR = KC / 2;            // lanes per row in a copy (16 bytes each)
  constexpr int RPI = 32 / LPR;          // rows per copy instruction
  constexpr int NCH = K / KC;            // stages per row group
  static_assert(K * N <= 1024, "B must fit in shared memory");
  const int64_t M = int64_t(1) << d.nm;
  const int64_t ulo = blockIdx.y % d.units_lo, uhi = blockIdx.y / d.units_lo;
  A += ulo * d.a_lo + uhi * d.a_hi;
  B += ulo * d.b_lo + uhi * d.b_hi;
  C += ulo * d.c_lo + uhi * d.c_hi;
  __shared__ __align__(16) float2 Bs[K * N];
  __shared__ __align__(16) float2 stage[SW][2][32 * PITCH];
  __shared__ int32_t nC[N];
  __shared__ int32_t tAlo[32], tAhi[32], tClo[32], tChi[32];
  __shared__ int32_t baseA, baseC;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t base = (int64_t)blockIdx.x * CH;
  for (int e = tid; e < K * N; e += SNT) {
    const int k = e / N, n = e % N;
    Bs[e] = B[bit_offset(k, NK, d.bk) + bit_offset(n, NN, d.bn)];
  }
  if (tid < N) nC[tid] = bit_offset(tid, NN, d.cn);
  const int lb = d.nm < CH_BITS ? d.nm : CH_BITS;
  if (tid >= 32 && tid < 64) {
    const int x = tid - 32;
    tAlo[x] = bit_offset(x, 5, d.am);  // lb >= 5
    tClo[x] = bit_offset(x, 5, d.cm);
  }
  if (tid >= 64 && tid < 96) {
    const int x = tid - 64, b1 = lb - 5;
    tAhi[x] = x < (1 << b1) ? bit_offset(x, b1, d.am + 5) : 0;
    tChi[x] = x < (1 << b1) ? bit_offset(x, b1, d.cm + 5) : 0;
  }
  if (tid == 96) {
    int32_t oa = 0, oc = 0;
    for (int i = CH_BITS; i < d.nm; ++i)
      if ((base >> i) & 1) { oa += d.am[i]; oc += d.cm[i]; }
    baseA = oa;
    baseC = oc;
  }
  __syncthreads();
  const int64_t rows = M - base < CH ? M - base : CH;
  const int ngroups = (int)(rows >> 5);
  const int nitems = ngroups > warp ? ((ngroups - 1 - warp) / SW + 1) * NCH : 0;
  float2* st = stage[warp][0];
  // copy of item i = (row group warp + SW (i / NCH), K chunk i % NCH) into buffer i & 1
  auto issue = [&](int i) {
    const int g = warp + SW * (i / NCH), c = i % NCH;
    const float2* src = A + baseA + tAhi[g] + (int64_t)c * KC + (lane % LPR) * 2;
    float2* dst = st + (i & 1) * 32 * PITCH + (lane % LPR) * 2;
#pragma unroll
    for (int q = 0; q < LPR; ++q) {
      const int r = q * RPI + lane / LPR;
      cp_async16(dst + r * PITCH, src + tAlo[r]);
    }
  };
  float2 acc[N];
#pragma unroll
  for (int n = 0; n < N; ++n) acc[n] = make_float2(0.f, 0.f);
  float mx = 0.f;
  if (nitems > 0) issue(0);
  cp_async_commit();
#pragma unroll 1
  for (int i = 0; i < nitems; ++i) {
    if (i + 1 < nitems) issue(i + 1);
    cp_async_commit();
    cp_async_wait1();
    __syncwarp();
    const int c = i % NCH;
    const float2* row = st + (i & 1) * 32 * PITCH + lane * PITCH;
#pragma unroll
    for (int kk = 0; kk < KC; kk += 2) {
      const float4 x = *reinterpret_cast<const float4*>(row + kk);
      const int k = c * KC + kk;
      mac_pair<N>(acc, Bs + k * N, Bs + (k + 1) * N, make_float2(x.x, x.y), make_float2(x.z, x.w));
    }
    __syncwarp();  // every lane is done with this buffer before it is refilled
    if (c == NCH - 1) {
      const int g = warp + SW * (i / NCH);
      const int32_t oc = baseC + tChi[g] + tClo[lane];
#pragma unroll
      for (int n = 0; n < N; ++n) {
        emit(o, C, (int64_t)oc + nC[n], acc[n], mx);
        acc[n] = make_float2(0.f, 0.f);
      }
    }
  }
  record_max(o.maxbits, mx);
}

// The staged kernel applies when A's K values of a row are contiguous, every
// copied 16-byte piece is aligned, and M >= 32.
bool staged_ok(const float2* A, const GemmDesc& d) {
  if (d.nk < 3 || d.nk > 7 || d.nm < 5 || (d.nk > 4 && d.nn > 3) || d.nn > 4) return false;
  if ((reinterpret_cast<uintptr_t>(A) & 15) != 0 || (d.a_lo & 1) != 0 || (d.a_hi & 1) != 0) return false;
  for (int i = 0; i < d.nk; ++i)
    if (d.ak[i] != (int32_t(1) << i)) return false;
  for (int i = 0; i < d.nm; ++i)
    if (d.am[i] & 1) return false;
  return true;
}

template <int NK>
cudaError_t launch_staged(const float2* A, const float2* B, float2* C, const GemmDesc& d, cudaStream_t s,
                          const VecOut& mb) {
  const dim3 g((unsigned)(((int64_t(1) << d.nm) + CH - 1) / CH), (unsigned)d.units);
  switch (d.nn) {
    case 0: vector_staged_kernel<NK, 0><<<g, SNT, 0, s>>>(A, B, C, d, mb); break;
    case 1: vector_staged_kernel<NK, 1><<<g, SNT, 0, s>>>(A, B, C, d, mb); break;
    case 2: vector_staged_kernel<NK, 2><<<g, SNT, 0, s>>>(A, B, C, d, mb); break;
    case 3: vector_staged_kernel<NK, 3><<<g, SNT, 0, s>>>(A, B, C, d, mb); break;
    case 4:
      if constexpr (NK <= 4) {
        vector_staged_kernel<NK, 4><<<g, SNT, 0, s>>>(A, B, C, d, mb);
        break;
      }
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int NK>
cudaError_t launch_long(const float2* A, const float2* B, float2* C, const GemmDesc& d, dim3 g, cudaStream_t s,
                        const VecOut& mb) {
  // pairs (k, k + 1), k even, are adjacent when A's K bit 0 has stride 1;
  // every other stride of A is then even, so a pair starts on a 16-byte
  // boundary once the base and the unit strides are even
  const int pair_k = d.nk >= 1 && d.ak[0] == 1 && (reinterpret_cast<uintptr_t>(A) & 15) == 0 &&
                     (d.a_lo & 1) == 0 && (d.a_hi & 1) == 0;
  switch (d.nn) {
    case 0: vector_long_kernel<NK, 0><<<g, NT, 0, s>>>(A, B, C, d, pair_k, mb); break;
    case 1: vector_long_kernel<NK, 1><<<g, NT, 0, s>>>(A, B, C, d, pair_k, mb); break;
    case 2: vector_long_kernel<NK, 2><<<g, NT, 0, s>>>(A, B, C, d, pair_k, mb); break;
    case 3: vector_long_kernel<NK, 3><<<g, NT, 0, s>>>(A, B, C, d, pair_k, mb); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int NK>
cudaError_t launch_nn(const float2* A, const float2* B, float2* C, const GemmDesc& d, dim3 g, cudaStream_t s,
                      const VecOut& mb) {
  switch (d.nn) {
    case 0: vector_kernel<NK, 0><<<g, NT, 0, s>>>(A, B, C, d, mb); break;
    case 1: vector_kernel<NK, 1><<<g, NT, 0, s>>>(A, B, C, d, mb); break;
    case 2: vector_kernel<NK, 2><<<g, NT, 0, s>>>(A, B, C, d, mb); break;
    case 3: vector_kernel<NK, 3><<<g, NT, 0, s>>>(A, B, C, d, mb); break;
    case 4: vector_kernel<NK, 4><<<g, NT, 0, s>>>(A, B, C, d, mb); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

bool vector_shape_ok(const GemmDesc& d) {
  return (d.nn <= 4 && d.nk <= 4) || (d.nn <= 3 && d.nk <= 7) || (d.nn <= 8 && d.nk <= 2) ||
         (d.nn == 5 && d.nk == 3);
}

// K = 8, N = 32: the tensor-core tile is 128 x 32 with one 16-K step (its upper
// half zeros), a few hundred cycles of MMA against an epilogue and pipeline
// round trip per tile; the streaming kernel does the 256 complex products per
// row on the FP32 cores at about the memory rate instead.
bool stream_preferred(const GemmDesc& d) { return d.nn == 5 && d.nk == 3; }

template <int NK>
cudaError_t launch_wide(const float2* A, const float2* B, float2* C, const GemmDesc& d, dim3 g, cudaStream_t s,
                        const VecOut& mb) {
  // pairs (k, k + 1), k even, adjacent and 16-byte aligned: A's K bit 0 has
  // stride 1 (every other stride of A is then even), even unit strides
  const int pair_k = NK >= 1 && d.ak[0] == 1 && (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (d.a_lo & 1) == 0 &&
                     (d.a_hi & 1) == 0;
  auto one = [&](auto nn) -> cudaError_t {
    constexpr int NN = decltype(nn)::value;
    if constexpr (((1 << NK) << NN) <= 1024) {
      vector_wide_kernel<NK, NN><<<g, NT, 0, s>>>(A, B, C, d, mb, pair_k);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  };
  switch (d.nn) {
    case 5: return one(std::integral_constant<int, 5>{});
    case 6: return one(std::integral_constant<int, 6>{});
    case 7: return one(std::integral_constant<int, 7>{});
    case 8: return one(std::integral_constant<int, 8>{});
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_vector(const float2* A, const float2* B, float2* C, const GemmDesc& d, cudaStream_t s,
                          const VecOut& maxbits) {
  if (!vector_shape_ok(d) || d.units > 65535) return cudaErrorInvalidValue;
  int64_t M = int64_t(1) << d.nm;
  dim3 g((unsigned)((M + CH - 1) / CH), (unsigned)d.units);
  if (d.nn == 5 && d.nk == 3) return launch_wide<3>(A, B, C, d, g, s, maxbits);
  if (d.nn > 4) {  // K <= 2 (vector_shape_ok)
    switch (d.nk) {
      case 0: return launch_wide<0>(A, B, C, d, g, s, maxbits);
      case 1: return launch_wide<1>(A, B, C, d, g, s, maxbits);
      default: return launch_wide<2>(A, B, C, d, g, s, maxbits);
    }
  }
  if (staged_ok(A, d)) {
    switch (d.nk) {
      case 3: return launch_staged<3>(A, B, C, d, s, maxbits);
      case 4: return launch_staged<4>(A, B, C, d, s, maxbits);
      case 5: return launch_staged<5>(A, B, C, d, s, maxbits);
      case 6: return launch_staged<6>(A, B, C, d, s, maxbits);
      default: return launch_staged<7>(A, B, C, d, s, maxbits);
    }
  }
  if (d.nk > 4) {
    switch (d.nk) {
      case 5: return launch_long<5>(A, B, C, d, g, s, maxbits);
      case 6: return launch_long<6>(A, B, C, d, g, s, maxbits);
      default: return launch_long<7>(A, B, C, d, g, s, maxbits);
    }
  }
  switch (d.nk) {
    case 0: return launch_nn<0>(A, B, C, d, g, s, maxbits);
    case 1: return launch_nn<1>(A, B, C, d, g, s, maxbits);
    case 2: return launch_nn<2>(A, B, C, d, g, s, maxbits);
    case 3: return launch_nn<3>(A, B, C, d, g, s, maxbits);
    default: return launch_nn<4>(A, B, C, d, g, s, maxbits);
  }
}

}  // namespace tn
