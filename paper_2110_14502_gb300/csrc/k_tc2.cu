// Warp-specialized tcgen05 GEMM fed by TMA, for complex operands prepared as
// four K-major 16-bit planes {re_hi, re_lo, im_hi, im_lo} (see k_split.cu).
//
// Paper: Sec. "Tensor Contraction Using Fused Permutation and Multiplication"
// (dense case: high compute density contraction at near-peak rate) and Sec.
// "A Mixed-Precision Computation Method via Adaptive Precision Scaling"
// (half-precision products, single-precision accumulation).
//
// Complex product on real tensor cores, planar form:
//   Dr = Ar Br - Ai Bi,  Di = Ar Bi + Ai Br,
// FP32 accumulation in TMEM (Dr and Di take TN columns each), the minus sign
// through the MMA's negate-A bit.  Split precision (four planes re_hi, re_lo,
// im_hi, im_lo) expands each real product X Y as Xhi Yhi + Xhi Ylo + Xlo Yhi
// and runs in gemm_tma_chunked, which bounds the tensor core's truncating
// accumulation to short chunks; single precision (two planes re, im) keeps
// one 16-bit product and runs in gemm_tma_kernel (one tile per CTA) or
// gemm_tma_persistent (one CTA per SM, double-buffered accumulators).
//
// Adaptive scaling (Sec. "A Mixed-Precision Computation Method via Adaptive
// Precision Scaling"): a plane tensor stores x 2^-e with a per-unit integer
// exponent e and records the largest stored component.  The GEMM predicts a
// bound 2 K maxA maxB on its stored output, picks r so that the bound stays
// below 2^15 (inside fp16 range), writes C 2^-(eA+eB+r) and records
// eC = eA + eB + r and the actual maximum.  A unit whose values turn
// non-finite, or whose operand maximum fell below 2^-10 (most of the 16-bit
// range lost to underflow), is flagged for the executor's filter.
//
// Roles (256 threads): warp 0 lane 0 issues TMA loads of one K stage (32
// complex K values of a 128-row A tile and a TN-row B tile, all four planes,
// 64-byte swizzled) into a ring of stages guarded by full/empty mbarriers;
// warp 1 lane 0 issues the tcgen05.mma instructions and commits each stage
// back to its empty barrier; warp 2 owns the TMEM allocation; warps 4-7 read
// the accumulators (tcgen05.ld) and write complex64 C through per-row and
// per-column offsets (the output permutation).  Every wait is bounded: on
// expiry the CTA records an error code and stops issuing work; before it
// leaves, the producer waits (bounded) for every TMA load it issued and the
// MMA warp for every MMA it issued, so no asynchronous copy or MMA still
// targets the CTA's shared memory or TMEM when it releases them.  Each CTA
// loads its own operand tiles from this GPU's memory (no clusters).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdlib>
#include <mutex>

#include "kernels.h"

namespace tn {

namespace {

constexpr int TM = 128;
constexpr int TKC = 32;                 // complex K per stage (64-byte rows of 16-bit values)
constexpr int NTHREADS = 256;
constexpr int SMEM_BUDGET = 196 * 1024;
constexpr long long kWaitLimit = 1ll << 24;  // default polls of a pipeline wait
constexpr long long kDrainLimit = 1ll << 24;  // polls of a wait for this CTA's own copies / MMAs on the way out
constexpr int GROUP_M_DEFAULT = 16;

template <int TN, int NP>
struct Cfg2 {
  static constexpr int A_STAGE = NP * TM * 64;    // NP planes of 128 rows x 64 bytes
  static constexpr int B_STAGE = NP * TN * 64;
  static constexpr int STAGE = A_STAGE + B_STAGE;
  static constexpr int NSTAGE = (SMEM_BUDGET / STAGE) < 6 ? (SMEM_BUDGET / STAGE) : 6;
  static constexpr int SMEM = NSTAGE * STAGE + 1024;
  // accumulator columns per tile: Dr, Di (TN each)
  static constexpr int ACC = 2 * TN;
  static constexpr uint32_t TMEM_COLS = ACC < 32 ? 32 : ACC;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Polls of every pipeline wait of the kernels below on this device (set by
// set_tc_wait_limit; 0 makes every pipeline wait give up at once).
__device__ long long g_wait_limit = kWaitLimit;

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

// One contiguous run of global memory into shared memory (16-byte aligned
// addresses, a multiple of 16 bytes), completing on the stage's barrier.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// K-major operand without swizzle: core matrices of 8 rows x 16 bytes, each
// 128 contiguous bytes; `lbo` bytes between the two core matrices of a 16-K
// step, `sbo` bytes between 8-row groups; swizzle mode 0.
__device__ __forceinline__ uint64_t plain_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// K-major, 64-byte swizzled operand: stride byte offset 512 (8 rows x 64 B),
// descriptor version 1 (bits 46-47), swizzle mode 4 = 64 B (bits 61-63).
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// kind::f16 instruction descriptor: FP32 accumulate, A/B 16-bit format
// (0 fp16, 1 bf16), optional negate-A (bit 13), K-major A and B, N >> 3 at
// bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc2(bool bf16, int M, int N, bool neg_a) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((neg_a ? 1u : 0u) << 13) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ int32_t bit_offset(int64_t x, int nb, const int32_t* st) {
  int32_t o = 0;
  for (int i = 0; i < nb; ++i)
    if ((x >> i) & 1) o += st[i];
  return o;
}

template <bool BF16>
__device__ __forceinline__ void split16(float x, uint16_t& hi, uint16_t& lo) {
  if (BF16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
  } else {
    const __half h = __float2half_rn(x);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
  }
}

// Both parts of re and im at once: x = hi + lo, hi = rn16(x), lo = rn16(x - hi)
// (the same roundings as split16), packed as the four planes of one element:
// .x = re_hi | re_lo << 16, .y = im_hi | im_lo << 16.
template <bool BF16>
__device__ __forceinline__ uint2 split_pair(float re, float im) {
  uint32_t hu, lu;
  if (BF16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(re - hf.x, im - hf.y);
    hu = *reinterpret_cast<const uint32_t*>(&h);
    lu = *reinterpret_cast<const uint32_t*>(&l);
  } else {
    const __half2 h = __floats2half2_rn(re, im);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(re - hf.x, im - hf.y);
    hu = *reinterpret_cast<const uint32_t*>(&h);
    lu = *reinterpret_cast<const uint32_t*>(&l);
  }
  return make_uint2(__byte_perm(hu, lu, 0x5410), __byte_perm(hu, lu, 0x7632));
}

template <bool BF16>
__device__ __forceinline__ uint16_t to16(float x) {
  if (BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
  return __half_as_ushort(__float2half_rn(x));
}

// Multiplication by 2^e for the exponent shifts of the scaled formats.  A
// power of two in the normal range multiplies exactly, so one multiply gives
// the correctly rounded x 2^e (the value ldexpf returns); shifts outside
// [-126, 127] go through ldexpf.
struct Pow2 {
  int e;
  float f;
  bool direct;
  __device__ explicit Pow2(int e_) {
    e = e_;
    direct = e_ >= -126 && e_ <= 127;
    f = __int_as_float((min(max(e_, -126), 127) + 127) << 23);
  }
  __device__ float operator()(float x) const { return direct ? x * f : ldexpf(x, e); }
};

// Number of leading tile column bits that are C's fastest indices in order
// (strides 1, 2, 4, ..): runs of 2^vb tile columns are contiguous in C.
__device__ __forceinline__ int vec_bits(const GemmDesc& d) {
  int v = 0;
  while (v < 4 && v < d.nn && d.cn[v] == (1 << v)) ++v;
  return v;
}

// One thread's 16 consecutive tile columns of one row as NP 16-bit planes:
// each contiguous run of 2^vb columns goes out as one store per plane (the
// run starts at a multiple of 2^vb elements: every other index of C has a
// larger stride).
template <int NP>
__device__ __forceinline__ void store_planes(uint16_t* P, int64_t plane, int64_t ro, const int32_t* col, int vb,
                                             const uint16_t (&h)[NP][16]) {
  auto pk = [&](int p, int j) { return (uint32_t)h[p][j] | ((uint32_t)h[p][j + 1] << 16); };
  if (vb >= 3) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int64_t o = ro + col[8 * r];
#pragma unroll
      for (int p = 0; p < NP; ++p)
        *reinterpret_cast<uint4*>(P + p * plane + o) =
            make_uint4(pk(p, 8 * r), pk(p, 8 * r + 2), pk(p, 8 * r + 4), pk(p, 8 * r + 6));
    }
  } else if (vb == 2) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t o = ro + col[4 * r];
#pragma unroll
      for (int p = 0; p < NP; ++p) *reinterpret_cast<uint2*>(P + p * plane + o) = make_uint2(pk(p, 4 * r), pk(p, 4 * r + 2));
    }
  } else if (vb == 1) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int64_t o = ro + col[2 * r];
#pragma unroll
      for (int p = 0; p < NP; ++p) *reinterpret_cast<uint32_t*>(P + p * plane + o) = pk(p, 2 * r);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int64_t o = ro + col[j];
#pragma unroll
      for (int p = 0; p < NP; ++p) P[p * plane + o] = h[p][j];
    }
  }
}

// The same stores from 16 packed elements (split_pair): plane 0 re_hi, 1 re_lo,
// 2 im_hi, 3 im_lo.
__device__ __forceinline__ uint32_t plane_pair(const uint2 (&e)[16], int p, int j) {
  const uint32_t a = p < 2 ? e[j].x : e[j].y, b = p < 2 ? e[j + 1].x : e[j + 1].y;
  return __byte_perm(a, b, (p & 1) ? 0x7632 : 0x5410);
}
__device__ __forceinline__ void store_planes4(uint16_t* P, int64_t plane, int64_t ro, const int32_t* col, int vb,
                                              const uint2 (&e)[16]) {
  if (vb >= 3) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int64_t o = ro + col[8 * r];
#pragma unroll
      for (int p = 0; p < 4; ++p)
        *reinterpret_cast<uint4*>(P + p * plane + o) = make_uint4(plane_pair(e, p, 8 * r), plane_pair(e, p, 8 * r + 2),
                                                                  plane_pair(e, p, 8 * r + 4), plane_pair(e, p, 8 * r + 6));
    }
  } else if (vb == 2) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t o = ro + col[4 * r];
#pragma unroll
      for (int p = 0; p < 4; ++p)
        *reinterpret_cast<uint2*>(P + p * plane + o) = make_uint2(plane_pair(e, p, 4 * r), plane_pair(e, p, 4 * r + 2));
    }
  } else if (vb == 1) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int64_t o = ro + col[2 * r];
#pragma unroll
      for (int p = 0; p < 4; ++p) *reinterpret_cast<uint32_t*>(P + p * plane + o) = plane_pair(e, p, 2 * r);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int64_t o = ro + col[j];
      P[o] = (uint16_t)(e[j].x & 0xffffu);
      P[plane + o] = (uint16_t)(e[j].x >> 16);
      P[2 * plane + o] = (uint16_t)(e[j].y & 0xffffu);
      P[3 * plane + o] = (uint16_t)(e[j].y >> 16);
    }
  }
}

// The same for complex64 output (two complex values per 16-byte store).
__device__ __forceinline__ void store_c64(float2* C, int64_t ro, const int32_t* col, int vb, const float* vr,
                                          const float* vi) {
  if (vb >= 1) {
    const int run = vb >= 4 ? 16 : (1 << vb);
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
      // pairs (j, j + 1) are contiguous; a new run starts every `run` columns
      float4* q = reinterpret_cast<float4*>(C + ro + col[j & ~(run - 1)]) + ((j & (run - 1)) >> 1);
      *q = make_float4(vr[j], vi[j], vr[j + 1], vi[j + 1]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) C[ro + col[j]] = make_float2(vr[j], vi[j]);
  }
}

template <int NREG>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t* v);
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// Producer's way out: wait (bounded) until the TMA loads of the last
// min(issued, ns) stages it filled have landed.  Earlier stages were waited
// for by the MMA warp before their slots were refilled; on the normal path
// these phases have completed already and every wait returns at once.
__device__ __forceinline__ void drain_loads(uint64_t* full, int ns, int64_t issued, int* err) {
  for (int64_t q = issued > ns ? issued - ns : 0; q < issued; ++q)
    if (!mbar_wait(&full[q % ns], (uint32_t)((q / ns) & 1), kDrainLimit)) {
      atomicExch(err, 9);
      return;
    }
}

template <int TN, bool BF16, int NP>
__global__ void __launch_bounds__(NTHREADS, 1)
    gemm_tma_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                    float2* __restrict__ C, const GemmDesc d, int kp, int a_zlo, int a_zhi, int b_zlo, int b_zhi,
                    int c_planes, const ScaleIO sio, int* __restrict__ err) {
  static_assert(NP == 2, "split precision runs in gemm_tma_chunked");
  using CF = Cfg2<TN, NP>;
  constexpr int A_STAGE = CF::A_STAGE;
  constexpr int NS = CF::NSTAGE;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[NS], empty[NS], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int32_t rowC[TM], colC[TN];
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long wl = g_wait_limit;
  const int64_t ulo = blockIdx.z % d.units_lo, uhi = blockIdx.z / d.units_lo;
  const int za_lo = a_zlo ? (int)ulo : 0, za_hi = a_zhi ? (int)uhi : 0;
  const int zb_lo = b_zlo ? (int)ulo : 0, zb_hi = b_zhi ? (int)uhi : 0;
  C += ulo * d.c_lo + uhi * d.c_hi;
  // exponents: stored operand = true * 2^-e; output scale 2^-r on top of 2^-(eA+eB)
  int ea = 0, eb = 0, r = 0;
  bool weak = false;
  if (sio.ea) {
    const int za = za_lo + za_hi * (a_zlo ? d.units_lo : 1), zb = zb_lo + zb_hi * (b_zlo ? d.units_lo : 1);
    ea = sio.ea[za];
    eb = sio.eb[zb];
    const float ma = sio.ma[za], mb = sio.mb[zb];
    weak = !(ma >= 0x1p-10f) || !(mb >= 0x1p-10f);
    const float bound = 2.f * ldexpf(ma * mb, d.nk);
    if (bound > 0.f && isfinite(bound)) {
      int x;
      frexpf(bound, &x);  // bound < 2^x
      r = x - 15;
    }
  }
  // Grouped raster: tiles run GROUP_M M-tiles at a time with the N-tiles
  // inside a group varying slowest, so concurrently resident CTAs share A row
  // blocks and re-read B tiles from L2 rather than DRAM.
  int m0, n0;
  {
    const int ntm = (int)((int64_t(1) << d.nm) / TM), ntn = (int)((int64_t(1) << d.nn) / TN);
    const int t = blockIdx.x;
    const int GM = d.group_m > 0 ? d.group_m : GROUP_M_DEFAULT;
    const int per_group = GM * ntn;
    const int g = t / per_group, r = t % per_group;
    const int gm = min(GM, ntm - g * GM);
    m0 = (g * GM + r % gm) * TM;
    n0 = (r / gm) * TN;
  }
  const int nkt = (kp + TKC - 1) / TKC;  // a short K (8, 16) is one stage; TMA zero-fills past K

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(CF::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (warp >= 4) {  // output offsets, computed while the main loop runs
    const int t = tid - 128;
    const int64_t M = int64_t(1) << d.nm, N = int64_t(1) << d.nn;
    rowC[t] = (m0 + t < M) ? bit_offset(m0 + t, d.nm, d.cm) : -1;
    for (int j = t; j < TN; j += 128) colC[j] = (n0 + j < N) ? bit_offset(n0 + j, d.nn, d.cn) : -1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---- TMA producer (one lane; the warp reconverges before the final barrier)
    int nis = 0;  // stages issued
    for (int kt = 0; lane == 0 && kt < nkt; ++kt) {
      const int s = kt % NS;
      if (kt >= NS && !mbar_wait(&empty[s], ((kt / NS) - 1) & 1, wl)) {
        atomicExch(err, 11);
        abort_flag = 1;
        break;
      }
      if (abort_flag) break;
      uint8_t* st = smem + s * CF::STAGE;
      mbar_expect_tx(&full[s], CF::STAGE);
      tma_load_5d(st, &mapA, &full[s], kt * TKC, m0, 0, za_lo, za_hi);
      tma_load_5d(st + A_STAGE, &mapB, &full[s], kt * TKC, n0, 0, zb_lo, zb_hi);
      ++nis;
    }
    if (lane == 0) drain_loads(full, NS, nis, err);
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer (one lane)
    constexpr uint32_t I = idesc2(BF16, TM, TN, false), IN = idesc2(BF16, TM, TN, true);
    const uint32_t dr = tmem, di = tmem + TN;
    int issued = 0;
    for (int kt = 0; lane == 0 && kt < nkt; ++kt) {
      const int s = kt % NS;
      if (!mbar_wait(&full[s], (kt / NS) & 1, wl)) {
        atomicExch(err, 12);
        abort_flag = 1;
        break;
      }
      if (abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a = smem_u32(smem + s * CF::STAGE);
      const uint32_t b = a + A_STAGE;
#pragma unroll
      for (int kk = 0; kk < TKC / 16; ++kk) {
        uint64_t A_[NP], B_[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          A_[p] = sw64_desc(a + p * (TM * 64) + kk * 32);
          B_[p] = sw64_desc(b + p * (TN * 64) + kk * 32);
        }
        const uint32_t acc = (kt | kk) ? 1u : 0u;
        // planes: 0 re, 1 im
        mma(dr, A_[0], B_[0], I, acc);
        mma(dr, A_[1], B_[1], IN, 1u);
        mma(di, A_[0], B_[1], I, acc);
        mma(di, A_[1], B_[0], I, 1u);
      }
      commit(&empty[s]);
      ++issued;
    }
    if (lane == 0) {
      if (issued > 0) {
        commit(&done);  // tracks every MMA issued above
        // the MMAs have finished with the stages and the accumulator before
        // this warp reaches the final barrier, whatever the epilogue saw
        if (!mbar_wait(&done, 0, kDrainLimit)) atomicExch(err, 15);
      } else if (nkt > 0) {
        atomicExch(err, 13);
      }
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ---- epilogue (whole warps: tcgen05.ld is warp-collective)
    const int q = warp & 3;
    bool ok = nkt > 0 && mbar_wait(&done, 0, wl);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && lane == 0 && nkt > 0) atomicExch(err, 14);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool go = __all_sync(0xffffffffu, ok && !abort_flag);
    if (go) {
      const int r_ = q * 32 + lane;
      const int32_t ro = rowC[r_];
      // the tile's first four column bits are C's four fastest indices: each
      // thread's 16 columns form one contiguous run (16-element aligned)
      const int vb = vec_bits(d);
      // plane output: stored = acc 2^-r; complex64 output: true value = acc 2^(eA+eB)
      const Pow2 sc(c_planes ? -r : ea + eb);
      float vmax = 0.f;
      bool bad = false;
#pragma unroll 1
      for (int c0 = 0; c0 < TN; c0 += 16) {
        uint32_t ur[16], ui[16];
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
        tmem_ld<16>(lane_base + (uint32_t)c0, ur);
        tmem_ld<16>(lane_base + (uint32_t)(TN + c0), ui);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float vr[16], vi[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float xr = __uint_as_float(ur[j]), xi = __uint_as_float(ui[j]);
          vr[j] = sc(xr);
          vi[j] = sc(xi);
        }
        // M and N are multiples of the tile and of 16: a chunk is all in or all out
        if (ro < 0 || colC[c0] < 0) continue;
        if (c_planes) {
          // output consumed by another tensor-core step: write its NP 16-bit
          // planes at the same offsets
          uint16_t* P = reinterpret_cast<uint16_t*>(C);
          const int64_t plane = int64_t(1) << (d.nm + d.nn);
          uint16_t h[NP][16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            vmax = fmaxf(vmax, fmaxf(fabsf(vr[j]), fabsf(vi[j])));
            bad |= !isfinite(vr[j]) || !isfinite(vi[j]);
            h[0][j] = to16<BF16>(vr[j]);
            h[1][j] = to16<BF16>(vi[j]);
          }
          store_planes<NP>(P, plane, ro, &colC[c0], vb, h);
        } else {
          store_c64(C, ro, &colC[c0], vb, vr, vi);
        }
      }
      if (sio.mc || sio.flag) {
        // per-unit bookkeeping: largest stored component, exponent, filter flag
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        bad = __any_sync(0xffffffffu, bad);
        const int zc = (int)blockIdx.z;
        if (lane == 0) {
          if (sio.mc && c_planes) atomicMax(sio.mc + zc, __float_as_uint(vmax));
          if (sio.ec && c_planes && q == 0 && blockIdx.x == 0) sio.ec[zc] = ea + eb + r;
          if (sio.flag && (bad || weak)) sio.flag[sio.flag_by_lo ? (int)ulo : zc] = 1;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CF::TMEM_COLS));
  }
}

// Persistent variant: one CTA per SM walks the (unit, tile) work items; the
// K-stage ring runs on across items, and two TMEM accumulator buffers let the
// epilogue warps drain item j while the MMA warp already accumulates item j+1.
template <int TN, bool BF16, int NP>
__global__ void __launch_bounds__(NTHREADS, 1)
    gemm_tma_persistent(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                        float2* __restrict__ C0, const GemmDesc d, int kp, int a_zlo, int a_zhi, int b_zlo,
                        int b_zhi, int c_planes, const ScaleIO sio, int* __restrict__ err) {
  static_assert(NP == 2, "split precision runs in gemm_tma_chunked");
  using CF = Cfg2<TN, NP>;
  constexpr int NS = CF::NSTAGE;
  constexpr int A_STAGE = CF::A_STAGE;
  constexpr uint32_t COLS = 2 * CF::TMEM_COLS;  // two accumulator buffers
  static_assert(COLS <= 512, "two accumulator buffers must fit in the 512 TMEM columns");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[NS], empty[NS], acc_full[2], acc_empty[2], mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ int32_t colC[2][TN];
  __shared__ volatile int abort_flag;
  __shared__ volatile int epi_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long wl = g_wait_limit;
  const int64_t first = blockIdx.x, stride = gridDim.x;
  const int ntm = (int)((int64_t(1) << d.nm) / TM), ntn = (int)((int64_t(1) << d.nn) / TN);
  const int tiles = ntm * ntn;
  const int64_t items = (int64_t)tiles * d.units;
  const int nkt = (kp + TKC - 1) / TKC;  // a short K (8, 16) is one stage; TMA zero-fills past K
  const int GM = d.group_m > 0 ? d.group_m : GROUP_M_DEFAULT;
  auto decode = [&](int64_t item, int& unit, int& m0, int& n0) {
    unit = (int)(item / tiles);
    const int t = (int)(item % tiles);
    const int per_group = GM * ntn;
    const int g = t / per_group, r = t % per_group;
    const int gm = min(GM, ntm - g * GM);
    m0 = (g * GM + r % gm) * TM;
    n0 = (r / gm) * TN;
  };

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], 128); }
    mbar_init(&mma_done, 1);
    abort_flag = 0;
    epi_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---- TMA producer: the stage ring continues across items
    int64_t g = 0;
    for (int64_t it = first; lane == 0 && it < items && !abort_flag; it += stride) {
      int unit, m0, n0;
      decode(it, unit, m0, n0);
      const int ulo = unit % d.units_lo, uhi = unit / d.units_lo;
      const int za_lo = a_zlo ? ulo : 0, za_hi = a_zhi ? uhi : 0;
      const int zb_lo = b_zlo ? ulo : 0, zb_hi = b_zhi ? uhi : 0;
      for (int kt = 0; kt < nkt; ++kt, ++g) {
        const int s = (int)(g % NS);
        if (g >= NS && !mbar_wait(&empty[s], (uint32_t)(((g / NS) - 1) & 1), wl)) {
          atomicExch(err, 21);
          abort_flag = 1;
          break;
        }
        uint8_t* st = smem + s * CF::STAGE;
        mbar_expect_tx(&full[s], CF::STAGE);
        tma_load_5d(st, &mapA, &full[s], kt * TKC, m0, 0, za_lo, za_hi);
        tma_load_5d(st + A_STAGE, &mapB, &full[s], kt * TKC, n0, 0, zb_lo, zb_hi);
      }
    }
    if (lane == 0) drain_loads(full, NS, g, err);  // g = stages issued
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer: item j accumulates into TMEM buffer j & 1
    constexpr uint32_t I = idesc2(BF16, TM, TN, false), IN = idesc2(BF16, TM, TN, true);
    int64_t g = 0, j = 0;
    for (int64_t it = first; lane == 0 && it < items && !abort_flag; it += stride, ++j) {
      const int b = (int)(j & 1);
      if (j >= 2 && !mbar_wait(&acc_empty[b], (uint32_t)(((j / 2) - 1) & 1), wl)) {
        atomicExch(err, 22);
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dr = tmem + (uint32_t)(b * CF::ACC), di = dr + TN;
      bool ok = true;
      for (int kt = 0; kt < nkt; ++kt, ++g) {
        const int s = (int)(g % NS);
        if (!mbar_wait(&full[s], (uint32_t)((g / NS) & 1), wl)) {
          atomicExch(err, 23);
          abort_flag = 1;
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a = smem_u32(smem + s * CF::STAGE);
        const uint32_t bb = a + A_STAGE;
#pragma unroll
        for (int kk = 0; kk < TKC / 16; ++kk) {
          uint64_t A_[NP], B_[NP];
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            A_[p] = sw64_desc(a + p * (TM * 64) + kk * 32);
            B_[p] = sw64_desc(bb + p * (TN * 64) + kk * 32);
          }
          const uint32_t acc = (kt | kk) ? 1u : 0u;
          // planes: 0 re, 1 im
          mma(dr, A_[0], B_[0], I, acc);
          mma(dr, A_[1], B_[1], IN, 1u);
          mma(di, A_[0], B_[1], I, acc);
          mma(di, A_[1], B_[0], I, 1u);
        }
        commit(&empty[s]);
      }
      commit(&acc_full[b]);  // also on an aborted item, so the epilogue's wait ends
      if (!ok) break;
    }
    // every MMA issued has finished reading shared memory and writing TMEM
    // before this warp reaches the final barrier
    if (lane == 0 && g > 0) {
      commit(&mma_done);
      if (!mbar_wait(&mma_done, 0, kDrainLimit)) atomicExch(err, 26);
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ---- epilogue: drain buffer j & 1 while the MMA warp fills the other
    const int q = warp & 3;
    const int t = tid - 128;
    int64_t j = 0;
    for (int64_t it = first; it < items; it += stride, ++j) {
      const int b = (int)(j & 1);
      int unit, m0, n0;
      decode(it, unit, m0, n0);
      const int ulo = unit % d.units_lo, uhi = unit / d.units_lo;
      for (int jj = t; jj < TN; jj += 128) colC[b][jj] = bit_offset(n0 + jj, d.nn, d.cn);
      const int32_t ro = bit_offset(m0 + q * 32 + lane, d.nm, d.cm);
      bool ok = mbar_wait(&acc_full[b], (uint32_t)((j / 2) & 1), wl);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok && lane == 0) {
        atomicExch(err, 24);
        abort_flag = 1;
        epi_fail = 1;
      }
      // colC of this item and any failure are visible to all 4 epilogue warps;
      // every epilogue thread has also finished item j-1 (so colC[b ^ 1] of
      // item j+1 can be written after this point)
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (epi_fail) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float2* C = C0 + (int64_t)ulo * d.c_lo + (int64_t)uhi * d.c_hi;
      int ea = 0, eb = 0, r = 0;
      bool weak = false;
      if (sio.ea) {
        const int za = (a_zlo ? ulo : 0) + (a_zhi ? uhi : 0) * (a_zlo ? d.units_lo : 1);
        const int zb = (b_zlo ? ulo : 0) + (b_zhi ? uhi : 0) * (b_zlo ? d.units_lo : 1);
        ea = sio.ea[za];
        eb = sio.eb[zb];
        const float ma = sio.ma[za], mb = sio.mb[zb];
        weak = !(ma >= 0x1p-10f) || !(mb >= 0x1p-10f);
        const float bound = 2.f * ldexpf(ma * mb, d.nk);
        if (bound > 0.f && isfinite(bound)) {
          int x;
          frexpf(bound, &x);
          r = x - 15;
        }
      }
      const int vb = vec_bits(d);
      const Pow2 sc(c_planes ? -r : ea + eb);
      float vmax = 0.f;
      bool bad = false;
      const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * CF::ACC);
#pragma unroll 1
      for (int c0 = 0; c0 < TN; c0 += 16) {
        uint32_t ur[16], ui[16];
        tmem_ld<16>(lane_base + (uint32_t)c0, ur);
        tmem_ld<16>(lane_base + (uint32_t)(TN + c0), ui);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float vr[16], vi[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          float xr = __uint_as_float(ur[jj]), xi = __uint_as_float(ui[jj]);
          vr[jj] = sc(xr);
          vi[jj] = sc(xi);
        }
        if (c_planes) {
          uint16_t* P = reinterpret_cast<uint16_t*>(C);
          const int64_t plane = int64_t(1) << (d.nm + d.nn);
          uint16_t h[NP][16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            vmax = fmaxf(vmax, fmaxf(fabsf(vr[jj]), fabsf(vi[jj])));
            bad |= !isfinite(vr[jj]) || !isfinite(vi[jj]);
            h[0][jj] = to16<BF16>(vr[jj]);
            h[1][jj] = to16<BF16>(vi[jj]);
          }
          store_planes<NP>(P, plane, ro, &colC[b][c0], vb, h);
        } else {
          store_c64(C, ro, &colC[b][c0], vb, vr, vi);
        }
      }
      // buffer b may be refilled once every epilogue thread has read it
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
      if (sio.mc || sio.flag) {
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
          if (sio.mc && c_planes) atomicMax(sio.mc + unit, __float_as_uint(vmax));
          if (sio.ec && c_planes && q == 0 && m0 == 0 && n0 == 0) sio.ec[unit] = ea + eb + r;
          if (sio.flag && (bad || weak)) sio.flag[sio.flag_by_lo ? ulo : unit] = 1;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS));
  }
}

// Staged output of the chunked kernel.  A warp's 32 x 16 sub-tile (lanes =
// tile row bits 0..4, columns = tile column bits 0..3) covers 512 elements of
// C; sorted by their C stride these 9 bits give each element a C-order index.
// When the output's fastest indices interleave row and column bits (neither
// the lanes nor a thread's columns form long contiguous runs), the warp writes
// its values to shared memory at their C-order index and reads them back in
// C order, consecutive lanes taking consecutive 16-byte pieces (2 complex64
// values, or 8 values of one 16-bit plane): the first `run` sorted strides
// are 1, 2, 4, .., so each store instruction writes runs of 2^run values.
// For 16-bit plane output the same staging also serves layouts whose
// contiguous run lies along the lanes (rows fastest), where each thread would
// otherwise store its values two bytes at a time.
constexpr int STAGE_SLOTS = 512 + 64;  // 8-byte slots per warp: 512 elements, 2 padding slots after every 16

struct StageMap {
  bool on;
  int lane_idx;        // this lane's bits of its elements' C-order index
  int rank_c[4];       // C-order rank of column bits 0..3
  int32_t off_c64;     // C offset of this lane's pair (C-order index 2 lane) in read-back step 0
  int32_t step_c64[3]; // C offset added by bits 0..2 of the complex64 read-back step
  int32_t off_pl;      // C offset of this lane's 8 values (C-order index 8 lane) in read-back step 0
  int32_t step_pl;     // C offset added by the second plane read-back step
};

__device__ __forceinline__ StageMap stage_map(const GemmDesc& d, int lane, int vb, bool planes) {
  StageMap m;
  int32_t st[9], sst[9];
  int rnk[9];
  for (int b = 0; b < 5; ++b) st[b] = d.cm[b];
  for (int b = 0; b < 4; ++b) st[5 + b] = d.cn[b];
  for (int b = 0; b < 9; ++b) {  // the strides of C's indices are distinct powers of two
    int r = 0;
    for (int o = 0; o < 9; ++o) r += st[o] < st[b];
    rnk[b] = r;
    sst[r] = st[b];
  }
  int run = 0;
  while (run < 9 && sst[run] == (1 << run)) ++run;
  int lane_run = 0;
  while (lane_run < 5 && d.cm[lane_run] == (1 << lane_run)) ++lane_run;
  // complex64: staged only where it lengthens the contiguous runs; planes
  // (2-byte values): also where it merely turns 2-, 4- or 8-byte stores into
  // 16-byte ones (a thread's columns give fewer than 8 contiguous values)
  m.on = planes ? run >= 3 && vb < 3 : run >= 3 && lane_run < 5 && vb < 4 && run > lane_run && run > vb;
  m.lane_idx = 0;
  for (int b = 0; b < 5; ++b) m.lane_idx |= ((lane >> b) & 1) << rnk[b];
  for (int b = 0; b < 4; ++b) m.rank_c[b] = rnk[5 + b];
  // read-back step t, lane l: complex64 pair l + 32 t (C-order index bits
  // 1..5 from the lane, 6..8 from t); plane group of 8 values l + 32 t (bits
  // 3..7 from the lane, bit 8 from t)
  m.off_c64 = 0;
  m.off_pl = 0;
  for (int b = 0; b < 5; ++b) {
    m.off_c64 += ((lane >> b) & 1) * sst[1 + b];
    m.off_pl += ((lane >> b) & 1) * sst[3 + b];
  }
  for (int b = 0; b < 3; ++b) m.step_c64[b] = sst[6 + b];
  m.step_pl = sst[8];
  return m;
}

__device__ __forceinline__ int stage_slot(int idx) { return idx + ((idx >> 4) << 1); }
static_assert(511 + (511 >> 4) * 2 < STAGE_SLOTS, "the last element's slot lies inside the warp's slots");

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

// Split precision, persistent, with chunked accumulation.  The tensor core
// adds into its FP32 accumulator with truncation, so over a long K the error
// grows linearly and is biased toward zero.  Here every chunk of `chunk` K
// stages starts a fresh accumulator, and the epilogue warps add the chunks
// with round-to-nearest FP32 adds, so the bias scales with the chunk length,
// not with K.
//
// TMEM holds two buffers of 2 TN columns (Dr, Di).  The CTA's t-th tile keeps
// its running sum R in buffer t & 1: its first chunk accumulates there
// directly; every later chunk accumulates in the other buffer P, which the
// epilogue folds into R (R += P, read P, read R, add, write R) and releases.
// After the last chunk the epilogue scales and stores R while the MMA warp
// already runs the next tile's first chunk in the other buffer (the next
// tile's R), so the MMA warp waits only for the folds, never for a store.
// K stages per chunk (32 complex K each): 16 unless TN_SPLIT_CHUNK says
// otherwise; the bias grows with the chunk length, so longer chunks trade
// accuracy for fewer folds.
int split_chunk() {
  static const int c = [] {
    const char* e = getenv("TN_SPLIT_CHUNK");
    const int v = e ? atoi(e) : 16;
    return v >= 1 && v <= 4096 ? v : 16;
  }();
  return c;
}

// Chunked kernel with EW epilogue warps (4 or 8): 128 + 32 EW threads.  Eight
// epilogue warps (two per TMEM lane quarter, taking alternate 16-column
// chunks) double the epilogue's latency hiding for output-bound steps; their
// staging buffers leave room for fewer operand stages.
template <int TN, int EW>
struct ChunkCfg {
  static constexpr int THREADS = 128 + 32 * EW;
  static constexpr int STAGE_BYTES = EW * STAGE_SLOTS * 8;
  static constexpr int BUDGET = EW == 4 ? SMEM_BUDGET : 227 * 1024 - STAGE_BYTES - 1024 - 4096;
  static constexpr int STAGE = Cfg2<TN, 4>::STAGE;
  static constexpr int NS = (BUDGET / STAGE) < 6 ? (BUDGET / STAGE) : 6;
  static constexpr int SMEM = NS * STAGE + 1024 + STAGE_BYTES;
  static_assert(NS >= 2, "at least two operand stages");
};

// Planes of one operand for K = 8 (16-byte rows): byte address of plane p,
// row r of the unit (zlo, zhi) = base + zlo st_lo + zhi st_hi + p plane + 16 r.
// A null base selects the tensor-map loads.
struct BulkPlanes {
  const uint8_t* base;
  int64_t st_lo, st_hi, plane;
};

template <int TN, bool BF16, int EW>
__global__ void __launch_bounds__(ChunkCfg<TN, EW>::THREADS, 1)
    gemm_tma_chunked(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                     float2* __restrict__ C0, const GemmDesc d, int kp, int a_zlo, int a_zhi, int b_zlo, int b_zhi,
                     int c_planes, const ScaleIO sio, int chunk, int fold, int* __restrict__ err,
                     const BulkPlanes ba, const BulkPlanes bb) {
  constexpr int NP = 4;
  using CF = Cfg2<TN, NP>;
  constexpr int NS = ChunkCfg<TN, EW>::NS;
  constexpr int NT = ChunkCfg<TN, EW>::THREADS;
  constexpr int ET = 32 * EW;  // epilogue threads
  constexpr int A_STAGE = CF::A_STAGE;
  constexpr uint32_t BUF = 2 * TN;  // columns of one buffer
  constexpr uint32_t COLS = 2 * BUF < 32 ? 32 : 2 * BUF;
  static_assert(2 * BUF <= 512, "two accumulator buffers must fit in TMEM");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[NS], empty[NS], acc_full[2], acc_empty[2], mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ int32_t colC[TN];
  __shared__ volatile int abort_flag;
  __shared__ volatile int epi_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long wl = g_wait_limit;
  const int64_t first = blockIdx.x, stride = gridDim.x;
  // fold > 1: `fold` consecutive hi units share A, and their N = 2^nn columns
  // side by side form the TN columns of one tile (so TN = fold * 2^nn)
  const int nsub = 1 << d.nn;
  const int ntm = (int)((int64_t(1) << d.nm) / TM), ntn = fold > 1 ? 1 : (int)((int64_t(1) << d.nn) / TN);
  const int tiles = ntm * ntn;
  const int64_t items = (int64_t)tiles * (d.units / fold);
  const int nkt = (kp + TKC - 1) / TKC;  // a short K (8, 16) is one stage; TMA zero-fills past K
  const int nch = (nkt + chunk - 1) / chunk;
  const int GM = d.group_m > 0 ? d.group_m : GROUP_M_DEFAULT;
  const bool items32 = items < (int64_t(1) << 31);
  auto decode = [&](int64_t item, int& unit, int& m0, int& n0) {
    int t;
    if (items32) {  // 32-bit division: a 64-bit one is a long dependent sequence
      unit = (int)((uint32_t)item / (uint32_t)tiles);
      t = (int)((uint32_t)item - (uint32_t)unit * (uint32_t)tiles);
    } else {
      unit = (int)(item / tiles);
      t = (int)(item % tiles);
    }
    const int per_group = GM * ntn;
    const int g = t / per_group, r = t % per_group;
    const int gm = min(GM, ntm - g * GM);
    m0 = (g * GM + r % gm) * TM;
    n0 = (r / gm) * TN;
  };

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], ET); }
    mbar_init(&mma_done, 1);
    abort_flag = 0;
    epi_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
  }
  // K = 8: each operand plane sits in a stage as its 16-byte rows (one bulk
  // copy) followed by as many zero bytes, the second core matrix of every
  // 16-K MMA step; the zeros are written once here
  const bool k8 = ba.base != nullptr;  // set by the host only for K = 8
  constexpr int A_PLANE8 = 2 * TM * 16, B_PLANE8 = 2 * TN * 16;
  if (k8) {
    for (int s = 0; s < NS; ++s) {
      uint8_t* st = smem + s * CF::STAGE;
      for (int i = tid; i < 4 * (TM * 16 / 16); i += NT) {
        const int p = i / (TM * 16 / 16), o = i % (TM * 16 / 16);
        reinterpret_cast<uint4*>(st + p * A_PLANE8 + TM * 16)[o] = make_uint4(0u, 0u, 0u, 0u);
      }
      for (int i = tid; i < 4 * (TN * 16 / 16); i += NT) {
        const int p = i / (TN * 16 / 16), o = i % (TN * 16 / 16);
        reinterpret_cast<uint4*>(st + A_STAGE + p * B_PLANE8 + TN * 16)[o] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor core's reads
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---- TMA producer: the stage ring runs on across items
    int64_t g = 0;
    for (int64_t it = first; lane == 0 && it < items && !abort_flag; it += stride) {
      int unit, m0, n0;
      decode(it, unit, m0, n0);
      const int ulo = unit % d.units_lo, uhi = (unit / d.units_lo) * fold;
      const int za_lo = a_zlo ? ulo : 0, za_hi = a_zhi ? uhi : 0;
      const int zb_lo = b_zlo ? ulo : 0, zb_hi = b_zhi ? uhi : 0;
      for (int kt = 0; kt < nkt; ++kt, ++g) {
        const int s = (int)(g % NS);
        if (g >= NS && !mbar_wait(&empty[s], (uint32_t)(((g / NS) - 1) & 1), wl)) {
          atomicExch(err, 31);
          abort_flag = 1;
          break;
        }
        uint8_t* st = smem + s * CF::STAGE;
        if (k8) {
          // four 2 KB runs of A's planes and four runs of B's (per folded unit)
          mbar_expect_tx(&full[s], 4 * TM * 16 + 4 * TN * 16);
          const uint8_t* ga = ba.base + za_lo * ba.st_lo + za_hi * ba.st_hi + (int64_t)m0 * 16;
#pragma unroll
          for (int p = 0; p < 4; ++p) bulk_load(st + p * A_PLANE8, ga + p * ba.plane, TM * 16, &full[s]);
          for (int f = 0; f < fold; ++f) {
            const uint8_t* gb = bb.base + zb_lo * bb.st_lo + (fold > 1 ? uhi + f : zb_hi) * bb.st_hi +
                                (int64_t)(fold > 1 ? 0 : n0) * 16;
            const int rows = fold > 1 ? nsub : TN;
#pragma unroll
            for (int p = 0; p < 4; ++p)
              bulk_load(st + A_STAGE + p * B_PLANE8 + f * rows * 16, gb + p * bb.plane, rows * 16, &full[s]);
          }
          continue;
        }
        mbar_expect_tx(&full[s], CF::STAGE);
        tma_load_5d(st, &mapA, &full[s], kt * TKC, m0, 0, za_lo, za_hi);
        if (fold == 1) {
          tma_load_5d(st + A_STAGE, &mapB, &full[s], kt * TKC, n0, 0, zb_lo, zb_hi);
        } else {
          // the B map's box is one plane of 2^nn rows: plane p of hi unit
          // uhi + f goes to rows f * 2^nn.. of plane p in the stage
          for (int f = 0; f < fold; ++f)
#pragma unroll
            for (int p = 0; p < NP; ++p)
              tma_load_5d(st + A_STAGE + (p * TN + f * nsub) * 64, &mapB, &full[s], kt * TKC, 0, p, zb_lo, uhi + f);
        }
      }
    }
    if (lane == 0) drain_loads(full, NS, g, err);  // g = stages issued
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer.  Chunk 0 of the t-th tile goes to buffer t & 1, later
    // chunks to the other one; the n-th use of a buffer (n >= 1) waits for
    // the epilogue's (n-1)-th release of it.
    constexpr uint32_t I = idesc2(BF16, TM, TN, false), IN = idesc2(BF16, TM, TN, true);
    int64_t g = 0, t = 0;
    uint32_t used[2] = {0u, 0u};
    bool ok = true;
    for (int64_t it = first; lane == 0 && ok && it < items && !abort_flag; it += stride, ++t) {
      const int rb = (int)(t & 1);
      for (int c = 0; c < nch && ok; ++c) {
        const int b = c == 0 ? rb : 1 - rb;
        if (used[b] >= 1 && !mbar_wait(&acc_empty[b], (used[b] - 1) & 1, wl)) {
          atomicExch(err, 32);
          abort_flag = 1;
          ok = false;
          break;
        }
        ++used[b];
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dr = tmem + (uint32_t)b * BUF, di = dr + TN;
        const int k0 = c * chunk, k1 = min(nkt, k0 + chunk);
        for (int kt = k0; kt < k1; ++kt, ++g) {
          const int s = (int)(g % NS);
          if (!mbar_wait(&full[s], (uint32_t)((g / NS) & 1), wl)) {
            atomicExch(err, 33);
            abort_flag = 1;
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a = smem_u32(smem + s * CF::STAGE);
          const uint32_t b0 = a + A_STAGE;
          const int nkk = k8 ? 1 : TKC / 16;  // K = 8: one 16-K step, its upper half zeros
#pragma unroll 2
          for (int kk = 0; kk < nkk; ++kk) {
            uint64_t A_[NP], B_[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
              if (k8) {
                A_[p] = plain_desc(a + p * A_PLANE8, TM * 16, 128);
                B_[p] = plain_desc(b0 + p * B_PLANE8, TN * 16, 128);
              } else {
                A_[p] = sw64_desc(a + p * (TM * 64) + kk * 32);
                B_[p] = sw64_desc(b0 + p * (TN * 64) + kk * 32);
              }
            }
            const uint32_t acc = (kt > k0 || kk) ? 1u : 0u;
            // planes: 0 re_hi, 1 re_lo, 2 im_hi, 3 im_lo; the chunk is short,
            // so the hi*lo + lo*hi terms share the hi*hi accumulator
            mma(dr, A_[0], B_[0], I, acc);
            mma(dr, A_[0], B_[1], I, 1u);
            mma(dr, A_[1], B_[0], I, 1u);
            mma(dr, A_[2], B_[2], IN, 1u);
            mma(dr, A_[2], B_[3], IN, 1u);
            mma(dr, A_[3], B_[2], IN, 1u);
            mma(di, A_[0], B_[2], I, acc);
            mma(di, A_[0], B_[3], I, 1u);
            mma(di, A_[1], B_[2], I, 1u);
            mma(di, A_[2], B_[0], I, 1u);
            mma(di, A_[2], B_[1], I, 1u);
            mma(di, A_[3], B_[0], I, 1u);
          }
          commit(&empty[s]);
        }
        commit(&acc_full[b]);  // also after an abort, so the epilogue's wait ends
      }
    }
    // every MMA issued has finished reading shared memory and writing TMEM
    // before this warp reaches the final barrier
    if (lane == 0 && g > 0) {
      commit(&mma_done);
      if (!mbar_wait(&mma_done, 0, kDrainLimit)) atomicExch(err, 36);
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ---- epilogue: fold chunks 1.. into R; after the last one, store R.
    // Warp 4 + e reads TMEM lane quarter q = warp % 4 (the hardware's rule)
    // and, with eight epilogue warps, every other 16-column chunk (h).
    const int e = warp - 4, q = warp & 3, h = e >> 2;
    constexpr int CS = 16 * (EW / 4);  // column stride between a warp's chunks
    const int tq = tid - 128;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const StageMap sm = stage_map(d, lane, vec_bits(d), c_planes != 0);
    float2* const slots = reinterpret_cast<float2*>(smem + NS * CF::STAGE) + e * STAGE_SLOTS;
    // the C-order index of (lane, jj) is lane_idx | (jj's bits at their ranks);
    // the two parts have disjoint bits, so their slots add
    const int lane_slot = stage_slot(sm.lane_idx);
    int cs[4];  // slot offset of column bit b alone
    for (int b = 0; b < 4; ++b) cs[b] = stage_slot(1 << sm.rank_c[b]);
    auto col_slot = [&](int jj) {
      return ((jj & 1) ? cs[0] : 0) + ((jj & 2) ? cs[1] : 0) + ((jj & 4) ? cs[2] : 0) + ((jj & 8) ? cs[3] : 0);
    };
    // C offset of the thread's row: its bits 0..6 (q * 32 + lane) once, the
    // tile's bits 7.. per item as a warp sum (lane b holds row bit b's stride)
    const int32_t ro_lo = bit_offset(q * 32 + lane, min(7, d.nm), d.cm);
    const int32_t my_cm = lane >= 7 && lane < d.nm ? d.cm[lane] : 0;
    int last_n0 = -1;
    // scaling and the maximum / filter tracking only where the formats need them
    const bool track = sio.mc != nullptr || sio.flag != nullptr;
    int64_t t = 0;
    uint32_t seen[2] = {0u, 0u};
    for (int64_t it = first; it < items; it += stride, ++t) {
      int unit, m0, n0;
      decode(it, unit, m0, n0);
      const int ulo = unit % d.units_lo, uhi = (unit / d.units_lo) * fold;
      // the column offsets change with the tile's first column only (the
      // barriers around each item order these writes against every read)
      if (n0 != last_n0) {
        for (int jj = tq; jj < TN; jj += ET) colC[jj] = bit_offset(fold > 1 ? (jj & (nsub - 1)) : n0 + jj, d.nn, d.cn);
        last_n0 = n0;
      }
      const int32_t ro = ro_lo + (int32_t)__reduce_add_sync(0xffffffffu, (uint32_t)(((m0 >> lane) & 1) ? my_cm : 0));
      float2* Cu = C0 + (int64_t)ulo * d.c_lo + (int64_t)uhi * d.c_hi;
      // Scaled formats: exponents of the operands of the tile's f-th unit (a
      // folded tile holds `fold` hi units side by side, f = column / 2^nn,
      // with A shared and B, C of their own) and the output shift r that keeps
      // the predicted bound 2 K maxA maxB below 2^15.
      auto unit_scale = [&](int f, int& ea, int& eb, int& r, bool& weak) {
        ea = eb = r = 0;
        weak = false;
        if (!sio.ea) return;
        const int za = (a_zlo ? ulo : 0) + (a_zhi ? uhi : 0) * (a_zlo ? d.units_lo : 1);
        const int zb = (b_zlo ? ulo : 0) + (b_zhi ? uhi + f : 0) * (b_zlo ? d.units_lo : 1);
        ea = sio.ea[za];
        eb = sio.eb[zb];
        const float ma = sio.ma[za], mb = sio.mb[zb];
        weak = !(ma >= 0x1p-10f) || !(mb >= 0x1p-10f);
        const float bound = 2.f * ldexpf(ma * mb, d.nk);
        if (bound > 0.f && isfinite(bound)) {
          int x;
          frexpf(bound, &x);
          r = x - 15;
        }
      };
      const int vb = vec_bits(d);
      const int gw = fold > 1 ? nsub : TN;  // tile columns of one unit
      const int rb = (int)(t & 1);
      const uint32_t R = tmem + lane_off + (uint32_t)rb * BUF, P = tmem + lane_off + (uint32_t)(1 - rb) * BUF;
      for (int c = 0; c < nch; ++c) {
        const int b = c == 0 ? rb : 1 - rb;
        bool ok = mbar_wait(&acc_full[b], seen[b] & 1, wl);
        ++seen[b];
        ok = __all_sync(0xffffffffu, ok);
        if (!ok && lane == 0) {
          atomicExch(err, 34);
          abort_flag = 1;
          epi_fail = 1;
        }
        // colC of this item and any failure visible to every epilogue warp
        asm volatile("bar.sync 1, %0;" ::"r"(ET) : "memory");
        if (epi_fail) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (c == 0) continue;  // the first chunk accumulated in R itself
#pragma unroll 1
        for (int c0 = 16 * h; c0 < TN; c0 += CS) {
          uint32_t pr[16], pi[16], rr[16], ri[16];
          tmem_ld<16>(P + (uint32_t)c0, pr);
          tmem_ld<16>(P + (uint32_t)(TN + c0), pi);
          tmem_ld<16>(R + (uint32_t)c0, rr);
          tmem_ld<16>(R + (uint32_t)(TN + c0), ri);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            rr[jj] = __float_as_uint(__uint_as_float(rr[jj]) + __uint_as_float(pr[jj]));
            ri[jj] = __float_as_uint(__uint_as_float(ri[jj]) + __uint_as_float(pi[jj]));
          }
          tmem_st16(R + (uint32_t)c0, rr);
          tmem_st16(R + (uint32_t)(TN + c0), ri);
        }
        // R complete before it is read again; P free for the next chunk
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[1 - rb])) : "memory");
      }
      if (epi_fail) break;
      float vmax = 0.f;
      bool bad = false, weak = false;
      int ea = 0, eb = 0, r = 0;
      Pow2 sc(0);
#pragma unroll 1
      for (int c0 = 16 * h; c0 < TN; c0 += CS) {
        // columns of a folded tile belong to hi unit uhi + c0 / 2^nn (N >= 16:
        // a 16-column chunk never straddles two units); the warp's first and
        // last chunks among a unit's gw columns open and close its records
        const int f = fold > 1 ? (c0 >> d.nn) : 0;
        if (c0 % gw < CS) {
          unit_scale(f, ea, eb, r, weak);
          sc = Pow2(c_planes ? -r : ea + eb);
          vmax = 0.f;
          bad = false;
        }
        float2* C = Cu + (int64_t)f * d.c_hi;
        uint32_t ur[16], ui[16];
        tmem_ld<16>(R + (uint32_t)c0, ur);
        tmem_ld<16>(R + (uint32_t)(TN + c0), ui);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float vr[16], vi[16];
        if (sc.direct && sc.f == 1.f) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            vr[jj] = __uint_as_float(ur[jj]);
            vi[jj] = __uint_as_float(ui[jj]);
          }
        } else {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            vr[jj] = sc(__uint_as_float(ur[jj]));
            vi[jj] = sc(__uint_as_float(ui[jj]));
          }
        }
        if (c_planes) {
          uint16_t* Pl = reinterpret_cast<uint16_t*>(C);
          const int64_t plane = int64_t(1) << (d.nm + d.nn);
          if (track) {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              vmax = fmaxf(vmax, fmaxf(fabsf(vr[jj]), fabsf(vi[jj])));
              bad |= !isfinite(vr[jj]) || !isfinite(vi[jj]);
            }
          }
          uint2 e[16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) e[jj] = split_pair<BF16>(vr[jj], vi[jj]);
          if (sm.on) {
            // planes of one element packed in one 8-byte slot, in C order
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) reinterpret_cast<uint2*>(slots)[lane_slot + col_slot(jj)] = e[jj];
            __syncwarp();
            const int64_t ob = (int64_t)__shfl_sync(0xffffffffu, ro, 0) + colC[c0] + sm.off_pl;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              // C-order values 8 (lane + 32 t) .. + 7, one uint2 slot (4 planes) each
              const uint4* src = reinterpret_cast<const uint4*>(slots) + stage_slot(8 * (lane + 32 * t)) / 2;
              uint2 v[8];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const uint4 x = src[u];
                v[2 * u] = make_uint2(x.x, x.y);
                v[2 * u + 1] = make_uint2(x.z, x.w);
              }
              const int64_t o = ob + (t ? sm.step_pl : 0);
#pragma unroll
              for (int pl = 0; pl < NP; ++pl) {
                auto pp = [&](int e0) {
                  const uint32_t a = pl < 2 ? v[e0].x : v[e0].y, b = pl < 2 ? v[e0 + 1].x : v[e0 + 1].y;
                  return __byte_perm(a, b, (pl & 1) ? 0x7632 : 0x5410);
                };
                *reinterpret_cast<uint4*>(Pl + pl * plane + o) = make_uint4(pp(0), pp(2), pp(4), pp(6));
              }
            }
            __syncwarp();
          } else {
            store_planes4(Pl, plane, ro, &colC[c0], vb, e);
          }
        } else if (sm.on) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) slots[lane_slot + col_slot(jj)] = make_float2(vr[jj], vi[jj]);
          __syncwarp();
          const int64_t ob = (int64_t)__shfl_sync(0xffffffffu, ro, 0) + colC[c0] + sm.off_c64;
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            // C-order values 2 (lane + 32 t) and the next one: two adjacent slots
            const float4 x = reinterpret_cast<const float4*>(slots)[stage_slot(2 * (lane + 32 * t)) / 2];
            const int32_t o = ((t & 1) ? sm.step_c64[0] : 0) + ((t & 2) ? sm.step_c64[1] : 0) +
                              ((t & 4) ? sm.step_c64[2] : 0);
            *reinterpret_cast<float4*>(C + ob + o) = x;
          }
          __syncwarp();
        } else {
          store_c64(C, ro, &colC[c0], vb, vr, vi);
        }
        if (c0 % gw + CS >= gw && (sio.mc || sio.flag)) {
          // the unit's columns are done: its largest stored component,
          // exponent and filter flag (launch unit ulo + (uhi + f) units_lo)
          const int un = fold > 1 ? ulo + (uhi + f) * d.units_lo : unit;
          for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
          const bool any_bad = __any_sync(0xffffffffu, bad);
          if (lane == 0) {
            if (sio.mc && c_planes) atomicMax(sio.mc + un, __float_as_uint(vmax));
            if (sio.ec && c_planes && q == 0 && m0 == 0 && n0 == 0) sio.ec[un] = ea + eb + r;
            if (sio.flag && (any_bad || weak)) sio.flag[sio.flag_by_lo ? ulo : un] = 1;
          }
        }
      }
      // R read out: the MMA warp may start a later tile's chunks in it
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[rb])) : "memory");
      // every epilogue thread is done with colC before the next item rewrites it
      asm volatile("bar.sync 1, %0;" ::"r"(ET) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// 5-D map over one operand's planes: [hi unit][lo unit][plane][row][k] of
// 16-bit values; box = 32 k x box_rows x box_planes x 1 x 1 (box_planes 0:
// all np planes).  A plane row holds K >= 8 values (16 bytes or more); when
// K < 32 the box reaches past it and the copy fills those K positions with
// zeros (the other operand's are zero as well, so the products vanish), and
// the stage still receives the box's full byte count.
bool encode_planes(CUtensorMap* map, const PlaneOperand& o, int box_rows, int box_planes = 0) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int64_t set = (int64_t)o.np * o.rows * o.kp * 2;  // bytes of one plane set
  cuuint64_t dims[5] = {(cuuint64_t)o.kp, (cuuint64_t)o.rows, (cuuint64_t)o.np, (cuuint64_t)o.nlo, (cuuint64_t)o.nhi};
  cuuint64_t strides[4] = {(cuuint64_t)(o.kp * 2), (cuuint64_t)(o.rows * o.kp * 2),
                           (cuuint64_t)(o.nlo > 1 ? o.st_lo : set), (cuuint64_t)(o.nhi > 1 ? o.st_hi : set)};
  cuuint32_t box[5] = {(cuuint32_t)TKC, (cuuint32_t)box_rows, (cuuint32_t)(box_planes > 0 ? box_planes : o.np), 1, 1};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 5, const_cast<uint16_t*>(o.base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int TN, bool BF16, int NP>
cudaError_t launch_cfg(const CUtensorMap& ma, const CUtensorMap& mb, float2* C, const GemmDesc& d, int kp,
                       const int z[4], int c_planes, const ScaleIO& sio, int* err, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tma_kernel<TN, BF16, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg2<TN, NP>::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t M = int64_t(1) << d.nm, N = int64_t(1) << d.nn;
  dim3 grid((unsigned)((M / TM) * (N / TN)), 1, (unsigned)d.units);
  gemm_tma_kernel<TN, BF16, NP><<<grid, NTHREADS, Cfg2<TN, NP>::SMEM, s>>>(ma, mb, C, d, kp, z[0], z[1], z[2], z[3],
                                                                           c_planes, sio, err);
  return cudaGetLastError();
}

// SM count of the current device (one CTA per SM for the persistent kernels).
int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 148;
}

template <int TN, bool BF16, int NP>
cudaError_t launch_persistent(const CUtensorMap& ma, const CUtensorMap& mb, float2* C, const GemmDesc& d, int kp,
                              const int z[4], int c_planes, const ScaleIO& sio, int* err, cudaStream_t s) {
  static bool attr = false;
  static int sms = 0;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tma_persistent<TN, BF16, NP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg2<TN, NP>::SMEM);
    if (e != cudaSuccess) return e;
    sms = sm_count();
    attr = true;
  }
  const int64_t M = int64_t(1) << d.nm, N = int64_t(1) << d.nn;
  const int64_t items = (M / TM) * (N / TN) * d.units;
  const unsigned grid = (unsigned)std::min<int64_t>(items, sms);
  gemm_tma_persistent<TN, BF16, NP><<<grid, NTHREADS, Cfg2<TN, NP>::SMEM, s>>>(ma, mb, C, d, kp, z[0], z[1], z[2],
                                                                              z[3], c_planes, sio, err);
  return cudaGetLastError();
}

template <int TN, bool BF16, int EW>
cudaError_t launch_chunked_ew(const CUtensorMap& ma, const CUtensorMap& mb, float2* C, const GemmDesc& d, int kp,
                              const int z[4], int c_planes, const ScaleIO& sio, int fold, int* err, cudaStream_t s,
                              const BulkPlanes& ba, const BulkPlanes& bb) {
  using CC = ChunkCfg<TN, EW>;
  static bool attr = false;
  static int sms = 0;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(gemm_tma_chunked<TN, BF16, EW>, cudaFuncAttributeMaxDynamicSharedMemorySize, CC::SMEM);
    if (e != cudaSuccess) return e;
    sms = sm_count();
    attr = true;
  }
  const int64_t M = int64_t(1) << d.nm, N = int64_t(1) << d.nn;
  const int64_t items = (M / TM) * (fold > 1 ? 1 : N / TN) * (d.units / fold);
  const int chunk = split_chunk();
  const unsigned grid = (unsigned)std::min<int64_t>(items, sms);
  gemm_tma_chunked<TN, BF16, EW><<<grid, CC::THREADS, CC::SMEM, s>>>(ma, mb, C, d, kp, z[0], z[1], z[2], z[3],
                                                                      c_planes, sio, chunk, fold, err, ba, bb);
  return cudaGetLastError();
}

// Eight epilogue warps where the epilogue dominates a tile (a short K, at
// most four operand stages, and tiles of 64 or 128 columns: each warp then
// still has two or more column chunks per tile), four where the main loop
// does and the extra operand stage matters.
template <int TN, bool BF16>
cudaError_t launch_chunked(const CUtensorMap& ma, const CUtensorMap& mb, float2* C, const GemmDesc& d, int kp,
                           const int z[4], int c_planes, const ScaleIO& sio, int fold, int* err, cudaStream_t s,
                           const BulkPlanes& ba, const BulkPlanes& bb) {
  const int nkt = (kp + TKC - 1) / TKC;
  if (TN >= 64 && nkt <= 4)
    return launch_chunked_ew<TN, BF16, 8>(ma, mb, C, d, kp, z, c_planes, sio, fold, err, s, ba, bb);
  return launch_chunked_ew<TN, BF16, 4>(ma, mb, C, d, kp, z, c_planes, sio, fold, err, s, ba, bb);
}

template <bool BF16, int NP>
cudaError_t launch_tn(int TNv, bool persistent, const CUtensorMap& ma, const CUtensorMap& mb, float2* C,
                      const GemmDesc& d, int kp, const int z[4], int cp, const ScaleIO& sio, int fold, int* err,
                      cudaStream_t s, const BulkPlanes& ba = BulkPlanes{}, const BulkPlanes& bb = BulkPlanes{}) {
  if constexpr (NP == 4) {
    // split precision always runs the chunked persistent kernel (accuracy)
    (void)persistent;
    switch (TNv) {
      case 128: return launch_chunked<128, BF16>(ma, mb, C, d, kp, z, cp, sio, fold, err, s, ba, bb);
      case 64: return launch_chunked<64, BF16>(ma, mb, C, d, kp, z, cp, sio, fold, err, s, ba, bb);
      case 32: return launch_chunked<32, BF16>(ma, mb, C, d, kp, z, cp, sio, fold, err, s, ba, bb);
      case 16: return launch_chunked<16, BF16>(ma, mb, C, d, kp, z, cp, sio, fold, err, s, ba, bb);
      default: return cudaErrorInvalidValue;
    }
  } else {
    if (persistent) {
      switch (TNv) {
        case 128: return launch_persistent<128, BF16, NP>(ma, mb, C, d, kp, z, cp, sio, err, s);
        case 64: return launch_persistent<64, BF16, NP>(ma, mb, C, d, kp, z, cp, sio, err, s);
        case 32: return launch_persistent<32, BF16, NP>(ma, mb, C, d, kp, z, cp, sio, err, s);
        case 16: return launch_persistent<16, BF16, NP>(ma, mb, C, d, kp, z, cp, sio, err, s);
        default: return cudaErrorInvalidValue;
      }
    }
    switch (TNv) {
      case 128: return launch_cfg<128, BF16, NP>(ma, mb, C, d, kp, z, cp, sio, err, s);
      case 64: return launch_cfg<64, BF16, NP>(ma, mb, C, d, kp, z, cp, sio, err, s);
      case 32: return launch_cfg<32, BF16, NP>(ma, mb, C, d, kp, z, cp, sio, err, s);
      case 16: return launch_cfg<16, BF16, NP>(ma, mb, C, d, kp, z, cp, sio, err, s);
      default: return cudaErrorInvalidValue;
    }
  }
}

}  // namespace

cudaError_t set_tc_wait_limit(long long polls) {
  const long long v = polls < 0 ? kWaitLimit : polls;
  return cudaMemcpyToSymbol(g_wait_limit, &v, sizeof v);
}

int tma_tile_n(const GemmDesc& d) {
  const int def = d.nn >= 7 ? 128 : (1 << d.nn);
  if (d.tile_n >= 16 && d.tile_n <= def) return d.tile_n;
  return def;
}

int64_t split_plane_elems(int nrow_bits, int nk_bits, int np) {
  const int64_t kp = int64_t(1) << nk_bits;  // K >= 8 (tensor-core shapes): rows of >= 16 bytes
  return np * (int64_t(1) << nrow_bits) * kp;
}

cudaError_t launch_gemm_tma(const PlaneOperand& a, const PlaneOperand& b, float2* C, bool c_planes, const GemmDesc& d,
                            bool bf16, const ScaleIO& sio, int* err, cudaStream_t s) {
  if (!tc_shape_ok(d) || d.units > 65535 || a.kp != b.kp || a.kp % 8 || a.np != b.np ||
      (a.np != 2 && a.np != 4))
    return cudaErrorInvalidValue;
  int TNv = tma_tile_n(d);
  // persistent CTAs pay off once there are several tiles per SM to overlap
  bool persistent = d.persistent == 1;
  if (d.persistent == 0) {
    const int64_t items = ((int64_t(1) << d.nm) / TM) * ((int64_t(1) << d.nn) / TNv) * d.units;
    persistent = items >= 2 * 148;
  }
  // Narrow N with A shared by the hi units (e.g. one slice-only tensor against
  // the bitstrings of a group): fold consecutive hi units into the columns of
  // one tile, so that the MMAs run 128 columns wide and A is read once for
  // all of them (split precision; with scaling, the epilogue takes each
  // unit's exponents for its own columns).
  int fold = 1;
  if (a.np == 4 && d.nn < 7 && a.nhi == 1 && b.nhi > 1 && d.units_lo > 0) {
    const int uh = d.units / d.units_lo;
    while (fold * 2 <= (128 >> d.nn) && uh % (fold * 2) == 0) fold *= 2;
    if (fold > 1) TNv = (1 << d.nn) * fold;
  }

  const int b_rows = fold > 1 ? (1 << d.nn) : TNv;
  CUtensorMap ma, mb;
  if (!encode_planes(&ma, a, TM) || !encode_planes(&mb, b, b_rows, fold > 1 ? 1 : 0)) return cudaErrorInvalidValue;
  const int kpi = (int)a.kp;
  const int z[4] = {a.nlo > 1, a.nhi > 1, b.nlo > 1, b.nhi > 1};
  const int cp = c_planes ? 1 : 0;
  if (a.np == 4) {
    // K = 8: the operands' 16-byte rows go by contiguous bulk copies (one per
    // plane) instead of tensor-map boxes of 16-byte rows; every address and
    // size must be a multiple of 16 bytes, else the tensor maps serve
    auto bulk = [](const PlaneOperand& o) {
      BulkPlanes q;
      q.base = reinterpret_cast<const uint8_t*>(o.base);
      q.st_lo = o.nlo > 1 ? o.st_lo : 0;
      q.st_hi = o.nhi > 1 ? o.st_hi : 0;
      q.plane = o.rows * o.kp * 2;
      return q;
    };
    BulkPlanes qa = bulk(a), qb = bulk(b);
    auto aligned = [](const BulkPlanes& q) {
      return (reinterpret_cast<uintptr_t>(q.base) % 16) == 0 && q.st_lo % 16 == 0 && q.st_hi % 16 == 0 &&
             q.plane % 16 == 0;
    };
    if (kpi != 8 || !aligned(qa) || !aligned(qb)) qa = qb = BulkPlanes{};
    return bf16 ? launch_tn<true, 4>(TNv, persistent, ma, mb, C, d, kpi, z, cp, sio, fold, err, s, qa, qb)
                : launch_tn<false, 4>(TNv, persistent, ma, mb, C, d, kpi, z, cp, sio, fold, err, s, qa, qb);
  }
  return bf16 ? launch_tn<true, 2>(TNv, persistent, ma, mb, C, d, kpi, z, cp, sio, 1, err, s)
              : launch_tn<false, 2>(TNv, persistent, ma, mb, C, d, kpi, z, cp, sio, 1, err, s);
}

}  // namespace tn
