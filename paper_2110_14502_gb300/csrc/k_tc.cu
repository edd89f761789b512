// Fused permute-GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Paper: Sec. "Tensor Contraction Using Fused Permutation and Multiplication"
// (dense case: fetch the permuted operand blocks and multiply them without a
// separate permutation pass) and Sec. "A Mixed-Precision Computation Method
// via Adaptive Precision Scaling" (half-precision products, single-precision
// accumulation).
//
// Complex arithmetic uses the real block form: with A' = [Ar | Ai] interleaved
// along K (A'[m][2k+c]) and B'[2k+c][2n+d] = {Br, Bi; -Bi, Br}[c][d],
// D'[m][2n+d] = sum A' B' gives (Cr, Ci) interleaved -- 8 real MMA flops per
// complex multiply-add, the counted rate.  For the split precision each
// operand is x = hi + lo with hi = rn16(x), lo = rn16(x - hi) and the product
// keeps hi*hi + hi*lo + lo*hi (three MMAs into the same FP32 accumulator).
// The tensor core adds into that accumulator with truncation, which over a
// long K leaves an error growing with K and biased toward zero; so each chunk
// of CHUNK K stages after the first accumulates into a fresh partial P, which
// all warps then add into the running sum R with round-to-nearest FP32 adds.
//
// Per CTA: one 128 (complex rows) x TN (complex columns) output tile held in
// TMEM as 128 lanes x 2 TN FP32 columns (R), plus 2 TN columns for P.  Each K stage of 32 complex values is
// gathered from global memory through per-row / per-column offsets (the
// permutation), converted to 16-bit hi/lo, and stored K-major in 128-byte
// swizzled shared memory; one thread issues the tcgen05.mma instructions and
// commits them to the stage's mbarrier, which the loaders wait on before they
// refill that stage.  Global loads of stage i+1 are issued before the MMAs of
// stage i are queued, so they overlap.  Every mbarrier wait is bounded: on
// expiry the CTA records an error word, skips the rest of its work and still
// releases its TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"

namespace tn {

namespace {

constexpr int TM = 128;          // complex rows per tile (= MMA M)
constexpr int TK = 32;           // complex K per stage (64 reals = one 128-byte swizzle row)
constexpr int NTHREADS = 256;
constexpr int A_TILE = 128 * 128;                   // 128 rows x 128 bytes
constexpr long long kWaitLimit = 1ll << 24;
constexpr int CHUNK = 16;        // K stages per TMEM partial sum

// Tile configuration by complex column count TN (MMA N = 2 TN reals).
template <int TN>
struct Cfg {
  static constexpr int B_TILE = 2 * TN * 128;                 // 2 TN rows x 128 bytes
  static constexpr int STAGE = 2 * A_TILE + 2 * B_TILE;       // A hi, A lo, B' hi, B' lo
  static constexpr int NSTAGE = TN == 64 ? 3 : 2;
  static constexpr int SMEM = NSTAGE * STAGE + 1024;          // + alignment slack
  static constexpr uint32_t TMEM_COLS = 4 * TN;               // running sum R and chunk partial P
  static constexpr int BCH = TN * 8 / NTHREADS;               // B chunks per thread
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the given phase parity; returns false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < kWaitLimit; ++it) {
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

// K-major, 128-byte swizzled operand descriptor (tcgen05 shared memory descriptor):
// start address >> 4 in bits 0-13, leading byte offset (unused for this
// layout) in 16-29, stride byte offset 1024 (8 rows x 128 B) in 32-45,
// descriptor version 1 in bits 46-47, swizzle mode 2 (128 B) in bits 61-63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B format (bits 7-9, 10-12: 0 fp16, 1 bf16), both K-major, N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_f16(bool bf16, int M, int N) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ int32_t bit_offset(int64_t x, int nb, const int32_t* st) {
  int32_t o = 0;
  for (int i = 0; i < nb; ++i)
    if ((x >> i) & 1) o += st[i];
  return o;
}

// Byte offset of 16-byte chunk `c` of row `r` in a 128-byte swizzled tile.
__device__ __forceinline__ uint32_t sw_off(int r, int c) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

template <bool BF16>
struct Half16;
template <>
struct Half16<true> {
  static __device__ __forceinline__ void split(float x, uint16_t& hi, uint16_t& lo) {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
  }
};
template <>
struct Half16<false> {
  static __device__ __forceinline__ void split(float x, uint16_t& hi, uint16_t& lo) {
    __half h = __float2half_rn(x);
    __half l = __float2half_rn(x - __half2float(h));
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(l);
  }
};

__device__ __forceinline__ uint32_t pack2(uint16_t a, uint16_t b) { return (uint32_t)a | ((uint32_t)b << 16); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

// Register staging of one K stage: each thread owns 4 A-chunks and BCH
// B-chunks, a chunk being 4 consecutive complex K values of one row (A) or
// column (B).
template <int BCH>
struct Stage {
  float2 a[4][4];
  float2 b[BCH][4];
};

template <bool BF16, int TN>
__global__ void __launch_bounds__(NTHREADS, 1)
    gemm_tc_kernel(const float2* __restrict__ A, const float2* __restrict__ B, float2* __restrict__ C,
                   const GemmDesc d, float a_scale, float b_scale, int* __restrict__ err) {
  using CF = Cfg<TN>;
  constexpr int NSTAGE = CF::NSTAGE, STAGE_BYTES = CF::STAGE, BCH = CF::BCH;
  constexpr uint32_t TMEM_COLS = CF::TMEM_COLS;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar_mma[NSTAGE];
  __shared__ uint64_t bar_done, bar_chunk;
  __shared__ uint32_t tmem_base_slot;
  __shared__ int32_t rowA[TM], rowC[TM], colB[TN], colC[TN];
  __shared__ int32_t kA[2][TK], kB[2][TK];
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t M = int64_t(1) << d.nm, N = int64_t(1) << d.nn, K = int64_t(1) << d.nk;
  const int64_t m0 = (int64_t)blockIdx.x * TM, n0 = (int64_t)blockIdx.y * TN;
  {
    const int64_t ulo = blockIdx.z % d.units_lo, uhi = blockIdx.z / d.units_lo;
    A += ulo * d.a_lo + uhi * d.a_hi;
    B += ulo * d.b_lo + uhi * d.b_hi;
    C += ulo * d.c_lo + uhi * d.c_hi;
  }
  if (tid < TM) {
    int64_t m = m0 + tid;
    rowA[tid] = m < M ? bit_offset(m, d.nm, d.am) : -1;
    rowC[tid] = m < M ? bit_offset(m, d.nm, d.cm) : -1;
  } else if (tid < TM + TN) {
    int64_t n = n0 + (tid - TM);
    colB[tid - TM] = n < N ? bit_offset(n, d.nn, d.bn) : -1;
    colC[tid - TM] = n < N ? bit_offset(n, d.nn, d.cn) : -1;
  }
  static_assert(TM + TN <= NTHREADS, "offset threads");
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) mbar_init(&bar_mma[s], 1);
    mbar_init(&bar_done, 1);
    mbar_init(&bar_chunk, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_slot)),
                 "r"(TMEM_COLS));  // 128 or 256 columns: a power of two >= 32
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  const int nkt = (int)((K + TK - 1) / TK);
  auto k_offsets = [&](int kt, int buf) {
    if (tid < TK) {
      int64_t k = (int64_t)kt * TK + tid;
      kA[buf][tid] = k < K ? bit_offset(k, d.nk, d.ak) : -1;
    } else if (tid >= 32 && tid < 32 + TK) {
      int64_t k = (int64_t)kt * TK + (tid - 32);
      kB[buf][tid - 32] = k < K ? bit_offset(k, d.nk, d.bk) : -1;
    }
  };
  k_offsets(0, 0);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_slot;

  // Chunk ownership.  A: 128 rows x 8 chunks = 1024 chunks, 4 per thread.
  // K-contiguous operands map consecutive threads to consecutive chunks of a
  // row; otherwise to consecutive rows (coalesced along M / N).
  const bool a_kfast = d.nk > 0 && d.ak[0] == 1;
  const bool b_kfast = d.nk > 0 && d.bk[0] == 1;
  // 4 consecutive K values contiguous in memory: one chunk = two 16-byte loads
  const bool a_vec = d.nk >= 2 && d.ak[0] == 1 && d.ak[1] == 2;
  const bool b_vec = d.nk >= 2 && d.bk[0] == 1 && d.bk[1] == 2;
  auto a_task = [&](int i, int& r, int& c) {
    int e = tid + i * NTHREADS;
    if (a_kfast) { r = e >> 3; c = e & 7; } else { r = e & 127; c = e >> 7; }
  };
  auto b_task = [&](int i, int& r, int& c) {  // B: TN columns x 8 chunks, BCH per thread
    int e = tid + i * NTHREADS;
    if (b_kfast) { r = e >> 3; c = e & 7; } else { r = e % TN; c = e / TN; }
  };
  auto load4 = [&](const float2* base, int32_t ro, const int32_t* ko, bool vec, float2* out) {
    if (vec) {
      // a chunk of 4 K values is either fully inside K or fully outside (K >= 4)
      if (ro >= 0 && ko[0] >= 0) {
        const float4* p = reinterpret_cast<const float4*>(base + (int64_t)ro + ko[0]);
        float4 x = __ldg(p), y = __ldg(p + 1);
        out[0] = make_float2(x.x, x.y); out[1] = make_float2(x.z, x.w);
        out[2] = make_float2(y.x, y.y); out[3] = make_float2(y.z, y.w);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) out[j] = make_float2(0.f, 0.f);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        out[j] = (ro >= 0 && ko[j] >= 0) ? __ldg(base + (int64_t)ro + ko[j]) : make_float2(0.f, 0.f);
    }
  };
  auto load_stage = [&](Stage<BCH>& st, int buf) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int r, c;
      a_task(i, r, c);
      load4(A, rowA[r], &kA[buf][c * 4], a_vec, st.a[i]);
    }
#pragma unroll
    for (int i = 0; i < BCH; ++i) {
      int r, c;
      b_task(i, r, c);
      load4(B, colB[r], &kB[buf][c * 4], b_vec, st.b[i]);
    }
  };
  auto store_stage = [&](const Stage<BCH>& st, int s) {
    uint8_t* base = smem + s * STAGE_BYTES;
    uint8_t* ahi = base;
    uint8_t* alo = base + A_TILE;
    uint8_t* bhi = base + 2 * A_TILE;
    uint8_t* blo = base + 2 * A_TILE + CF::B_TILE;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int r, c;
      a_task(i, r, c);
      uint16_t h[8], l[8];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        Half16<BF16>::split(st.a[i][j].x * a_scale, h[2 * j], l[2 * j]);
        Half16<BF16>::split(st.a[i][j].y * a_scale, h[2 * j + 1], l[2 * j + 1]);
      }
      const uint32_t o = sw_off(r, c);
      *(uint4*)(ahi + o) = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
      *(uint4*)(alo + o) = make_uint4(pack2(l[0], l[1]), pack2(l[2], l[3]), pack2(l[4], l[5]), pack2(l[6], l[7]));
    }
#pragma unroll
    for (int i = 0; i < BCH; ++i) {
      int r, c;
      b_task(i, r, c);
      // row 2r:   [Br, -Bi] per k;  row 2r+1: [Bi, Br] per k
      uint16_t rh[8], ih[8], nih[8], rl[8], il[8], nil[8];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint16_t h, l;
        Half16<BF16>::split(st.b[i][j].x * b_scale, h, l);
        rh[j] = h; rl[j] = l;
        Half16<BF16>::split(st.b[i][j].y * b_scale, h, l);
        ih[j] = h; il[j] = l;
        nih[j] = h ^ 0x8000; nil[j] = l ^ 0x8000;
      }
      const uint32_t o0 = sw_off(2 * r, c), o1 = sw_off(2 * r + 1, c);
      *(uint4*)(bhi + o0) = make_uint4(pack2(rh[0], nih[0]), pack2(rh[1], nih[1]), pack2(rh[2], nih[2]), pack2(rh[3], nih[3]));
      *(uint4*)(bhi + o1) = make_uint4(pack2(ih[0], rh[0]), pack2(ih[1], rh[1]), pack2(ih[2], rh[2]), pack2(ih[3], rh[3]));
      *(uint4*)(blo + o0) = make_uint4(pack2(rl[0], nil[0]), pack2(rl[1], nil[1]), pack2(rl[2], nil[2]), pack2(rl[3], nil[3]));
      *(uint4*)(blo + o1) = make_uint4(pack2(il[0], rl[0]), pack2(il[1], rl[1]), pack2(il[2], rl[2]), pack2(il[3], rl[3]));
    }
  };

  constexpr uint32_t IDESC = idesc_f16(BF16, 128, 2 * TN);
  Stage<BCH> st;
  load_stage(st, 0);
  uint32_t nfold = 0;
  for (int kt = 0; kt < nkt; ++kt) {
    const int s = kt % NSTAGE;
    if (kt >= NSTAGE) {
      if (!mbar_wait(&bar_mma[s], ((kt / NSTAGE) - 1) & 1)) {
        atomicExch(err, 1);
        abort_flag = 1;
      }
    }
    __syncthreads();
    if (abort_flag) break;
    store_stage(st, s);
    if (kt + 1 < nkt) k_offsets(kt + 1, (kt + 1) & 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t ahi = sw128_desc(base + kk * 32);
        const uint64_t alo = sw128_desc(base + A_TILE + kk * 32);
        const uint64_t bhi = sw128_desc(base + 2 * A_TILE + kk * 32);
        const uint64_t blo = sw128_desc(base + 2 * A_TILE + CF::B_TILE + kk * 32);
        // chunk 0 accumulates into R, later chunks into a fresh P
        const uint32_t dst = kt < CHUNK ? tmem : tmem + 2 * TN;
        const uint32_t first = (kt % CHUNK == 0 && kk == 0) ? 0u : 1u;
        mma_f16(dst, ahi, bhi, IDESC, first);
        mma_f16(dst, ahi, blo, IDESC, 1u);
        mma_f16(dst, alo, bhi, IDESC, 1u);
      }
      mma_commit(&bar_mma[s]);
      if (kt >= CHUNK && (kt % CHUNK == CHUNK - 1 || kt == nkt - 1)) mma_commit(&bar_chunk);
      if (kt == nkt - 1) mma_commit(&bar_done);
    }
    if (kt + 1 < nkt) load_stage(st, (kt + 1) & 1);  // in flight while the MMAs above run
    if (kt >= CHUNK && (kt % CHUNK == CHUNK - 1 || kt == nkt - 1)) {
      // fold the chunk's partial P into R: warp w owns TMEM lanes 32 (w % 4)..
      // and half w / 4 of the 2 TN columns
      const bool ok = mbar_wait(&bar_chunk, nfold & 1);
      ++nfold;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(err, 3);
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int q = warp & 3, half = warp >> 2;
      const uint32_t lb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * TN);
#pragma unroll 1
      for (int cc = 0; cc < TN; cc += 16) {
        uint32_t pv[16], rv[16];
        tmem_ld16(lb + 2 * TN + cc, pv);
        tmem_ld16(lb + cc, rv);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) rv[j] = __float_as_uint(__uint_as_float(rv[j]) + __uint_as_float(pv[j]));
        tmem_st16(lb + cc, rv);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
  }
  __syncthreads();
  // On an aborted loop the last commit was never issued: commit now so that the
  // wait below also covers the MMAs already queued before TMEM is released.
  const bool aborted = abort_flag != 0;
  if (aborted && tid == 0 && nkt > 0) mma_commit(&bar_done);
  bool drained = true;
  if (nkt > 0 && !mbar_wait(&bar_done, 0)) {
    atomicExch(err, 2);
    drained = false;
  }
  __syncthreads();
  if (!drained) abort_flag = 1;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!abort_flag) {
    // epilogue: warp w reads lanes 32*(w%4).. of TMEM; warps 0-3 take the
    // first half of the 2*TN columns, warps 4-7 the second half.
    const int q = warp & 3, half = warp >> 2;
    const int r = q * 32 + lane;
    const float inv = 1.0f / (a_scale * b_scale);
#pragma unroll
    for (int cc = 0; cc < TN / 32; ++cc) {
      const int col = half * TN + cc * 32;
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int32_t ro = rowC[r];
      if (ro >= 0) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int cn = col / 2 + j;
          const int32_t co = colC[cn];
          if (co >= 0) C[(int64_t)ro + co] = make_float2(__uint_as_float(v[2 * j]) * inv, __uint_as_float(v[2 * j + 1]) * inv);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace

bool tc_shape_ok(const GemmDesc& d) { return d.nm >= 7 && d.nn >= 4 && d.nk >= 3; }

template <bool BF16, int TN>
static cudaError_t launch_cfg(const float2* A, const float2* B, float2* C, const GemmDesc& d, float as, float bs,
                              int* err, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<BF16, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg<TN>::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t M = int64_t(1) << d.nm, N = int64_t(1) << d.nn;
  dim3 grid((unsigned)(M / TM), (unsigned)((N + TN - 1) / TN), (unsigned)d.units);
  gemm_tc_kernel<BF16, TN><<<grid, NTHREADS, Cfg<TN>::SMEM, s>>>(A, B, C, d, as, bs, err);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc(const float2* A, const float2* B, float2* C, const GemmDesc& d, bool bf16, float a_scale,
                           float b_scale, int* err, cudaStream_t s) {
  if (!tc_shape_ok(d) || d.units > 65535) return cudaErrorInvalidValue;
  const bool wide = d.nn >= 7;  // N >= 128 complex columns
  if (bf16) return wide ? launch_cfg<true, 128>(A, B, C, d, a_scale, b_scale, err, s)
                        : launch_cfg<true, 64>(A, B, C, d, a_scale, b_scale, err, s);
  return wide ? launch_cfg<false, 128>(A, B, C, d, a_scale, b_scale, err, s)
              : launch_cfg<false, 64>(A, B, C, d, a_scale, b_scale, err, s);
}

}  // namespace tn
