// Fused permute-GEMM on FP32 CUDA cores (complex64 in, complex64 out): the
// plain complex64 path, FP32 products and sums, no tensor cores.
//
// Paper: Sec. "Tensor Contraction Using Fused Permutation and Multiplication",
// dense case: the permutation of each operand is folded into the fetch of its
// tile rather than run as a separate pass.  Every element offset comes from
// the operand's per-bit strides (the analogue of the paper's pre-computed
// position array): a row's offset is computed once per CTA, and a K offset
// splits into the chunk's high bits (once per chunk) plus a per-thread
// constant for the low four bits.
//
// Tiling: a CTA of 256 threads computes a 128 x BN tile of C (BN = 64 or 128)
// over K chunks of 16.  Each thread owns an 8-row x (BN / 16)-column complex
// micro-tile: per chunk and k it reads 8 A values (4 x 16-byte shared loads,
// broadcast across the warp) and BN/16 B values, and issues 8 * BN/16 complex
// multiply-adds of 4 FFMA each.  The tiles are staged in shared memory k-major
// ([k][row], rows contiguous) with two buffers: the global loads of chunk c+1
// are in flight in registers while chunk c is computed, then stored to the
// other buffer; one barrier per chunk.
//
// Global loads: when the operand's two fastest indices are its first two K
// bits (the planner's layouts put contracted indices innermost), a thread
// reads 4 consecutive K values of one row as two 16-byte loads and the 32
// lanes of a warp read 32 rows at the same K quad (one 32-byte sector per
// row); otherwise each lane reads one element, lanes on consecutive rows.
#include "kernels.h"

namespace tn {

namespace {

constexpr int BM = 128, BK = 16, NT = 256;

__device__ __forceinline__ int32_t bit_offset(int64_t x, int nb, const int32_t* st) {
  int32_t o = 0;
  for (int i = 0; i < nb; ++i)
    if ((x >> i) & 1) o += st[i];
  return o;
}

// Offset of the K bits at and above bit 4 of k0 (a multiple of 16).
__device__ __forceinline__ int32_t k_high_offset(int64_t k0, int nk, const int32_t* st) {
  int32_t o = 0;
  for (int i = 4; i < nk; ++i)
    if ((k0 >> i) & 1) o += st[i];
  return o;
}

// One operand tile of R rows (128 or 64) x 16 K values: what this thread
// loads, where from and where it goes in shared memory.
template <int R>
struct TileLoader {
  static constexpr int NQ = R / 64;        // K quads per thread (vector path)
  static constexpr int NE = R / 16;        // elements per thread (scalar path)
  static constexpr int STEP = NT / R;      // K distance between a thread's scalar elements
  bool vec;
  int64_t K;
  int kq;                 // vector path: K quad of this thread
  int32_t row_off[NQ > 0 ? NQ : 1];
  int row[NQ > 0 ? NQ : 1];
  int32_t low_q;          // offset of K = 4 kq within a chunk
  int srow;               // scalar path: this thread's row
  int32_t srow_off;
  int32_t low_s[NE];      // offsets of K = kk0 + STEP j within a chunk
  int kk0;
  float2 v[NE];           // staged values (vector path: quad q's 4 values at 4 q ..)

  __device__ void init(const GemmDesc& d, int nrow_bits, const int32_t* rst, const int32_t* kst, int64_t r0,
                       bool vector_ok) {
    const int t = threadIdx.x;
    K = int64_t(1) << d.nk;
    const int64_t nrows = int64_t(1) << nrow_bits;
    vec = vector_ok;
    if (vec) {
      kq = (t >> 5) & 3;
      low_q = bit_offset(4 * kq, d.nk < 4 ? d.nk : 4, kst);
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        row[q] = (t & 31) + 32 * (t >> 7) + 64 * q;
        row_off[q] = r0 + row[q] < nrows ? bit_offset(r0 + row[q], nrow_bits, rst) : -1;
      }
    } else {
      srow = t % R;
      kk0 = t / R;
      srow_off = r0 + srow < nrows ? bit_offset(r0 + srow, nrow_bits, rst) : -1;
#pragma unroll
      for (int j = 0; j < NE; ++j) low_s[j] = bit_offset(kk0 + STEP * j, d.nk < 4 ? d.nk : 4, kst);
    }
  }

  __device__ __forceinline__ void load(const float2* __restrict__ src, int64_t k0, int32_t khi) {
    if (vec) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = x;
        if (row_off[q] >= 0 && k0 + 4 * kq < K) {
          const float4* p = reinterpret_cast<const float4*>(src + row_off[q] + khi + low_q);
          x = __ldg(p);
          y = __ldg(p + 1);
        }
        v[4 * q + 0] = make_float2(x.x, x.y);
        v[4 * q + 1] = make_float2(x.z, x.w);
        v[4 * q + 2] = make_float2(y.x, y.y);
        v[4 * q + 3] = make_float2(y.z, y.w);
      }
    } else {
#pragma unroll
      for (int j = 0; j < NE; ++j) {
        float2 x = make_float2(0.f, 0.f);
        if (srow_off >= 0 && k0 + kk0 + STEP * j < K) x = __ldg(src + srow_off + khi + low_s[j]);
        v[j] = x;
      }
    }
  }

  // tile [BK][R] in shared memory
  __device__ __forceinline__ void store(float2* tile) const {
    if (vec) {
#pragma unroll
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int j = 0; j < 4; ++j) tile[(4 * kq + j) * R + row[q]] = v[4 * q + j];
    } else {
#pragma unroll
      for (int j = 0; j < NE; ++j) tile[(kk0 + STEP * j) * R + srow] = v[j];
    }
  }
};

// flags: bit 0 A vector loads, bit 1 B vector loads, bit 2 C pair stores
template <int BN>
__global__ void __launch_bounds__(NT, 1) gemm_simt_kernel(const float2* __restrict__ A,
                                                           const float2* __restrict__ B,
                                                           float2* __restrict__ C, const GemmDesc d, int flags) {
  constexpr int WN = BN / 16;  // complex columns per thread
  extern __shared__ __align__(16) float2 smem[];
  float2* As = smem;                 // [2][BK][BM]
  float2* Bs = smem + 2 * BK * BM;   // [2][BK][BN]
  const int64_t K = int64_t(1) << d.nk;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int64_t ulo = blockIdx.z % d.units_lo, uhi = blockIdx.z / d.units_lo;
  A += ulo * d.a_lo + uhi * d.a_hi;
  B += ulo * d.b_lo + uhi * d.b_hi;
  C += ulo * d.c_lo + uhi * d.c_hi;
  const int tid = threadIdx.x;
  const int tn = tid & 15, tm = tid >> 4;  // 16 column groups x 16 row groups

  TileLoader<BM> la;
  TileLoader<BN> lb;
  la.init(d, d.nm, d.am, d.ak, m0, (flags & 1) != 0);
  lb.init(d, d.nn, d.bn, d.bk, n0, (flags & 2) != 0);

  float accr[8][WN], acci[8][WN];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < WN; ++j) accr[i][j] = acci[i][j] = 0.f;

  const int64_t nch = (K + BK - 1) / BK;
  la.load(A, 0, 0);
  lb.load(B, 0, 0);
  la.store(As);
  lb.store(Bs);
  __syncthreads();
  for (int64_t c = 0; c < nch; ++c) {
    const int buf = (int)(c & 1);
    if (c + 1 < nch) {
      const int64_t k1 = (c + 1) * BK;
      la.load(A, k1, k_high_offset(k1, d.nk, d.ak));
      lb.load(B, k1, k_high_offset(k1, d.nk, d.bk));
    }
    const float2* at = As + buf * BK * BM;
    const float2* bt = Bs + buf * BK * BN;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float ar[8], ai[8], br[WN], bi[WN];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 x = *reinterpret_cast<const float4*>(at + kk * BM + 8 * tm + 2 * i);
        ar[2 * i] = x.x;
        ai[2 * i] = x.y;
        ar[2 * i + 1] = x.z;
        ai[2 * i + 1] = x.w;
      }
#pragma unroll
      for (int j = 0; j < WN / 2; ++j) {
        // columns 2 tn, 2 tn + 1 of each 32-column band
        const float4 x = *reinterpret_cast<const float4*>(bt + kk * BN + 32 * j + 2 * tn);
        br[2 * j] = x.x;
        bi[2 * j] = x.y;
        br[2 * j + 1] = x.z;
        bi[2 * j + 1] = x.w;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < WN; ++j) {
          accr[i][j] = fmaf(ar[i], br[j], accr[i][j]);
          accr[i][j] = fmaf(-ai[i], bi[j], accr[i][j]);
          acci[i][j] = fmaf(ar[i], bi[j], acci[i][j]);
          acci[i][j] = fmaf(ai[i], br[j], acci[i][j]);
        }
    }
    if (c + 1 < nch) {
      la.store(As + (buf ^ 1) * BK * BM);
      lb.store(Bs + (buf ^ 1) * BK * BN);
    }
    __syncthreads();
  }

  // epilogue: C offsets of this thread's rows and columns
  const int64_t M = int64_t(1) << d.nm, N = int64_t(1) << d.nn;
  int32_t cc[WN];
#pragma unroll
  for (int j = 0; j < WN; ++j) {
    const int64_t n = n0 + 32 * (j >> 1) + 2 * tn + (j & 1);
    cc[j] = n < N ? bit_offset(n, d.nn, d.cn) : -1;
  }
  const bool pairs = (flags & 4) != 0;  // columns 2 tn, 2 tn + 1 adjacent in C (16-byte store)
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t m = m0 + 8 * tm + i;
    if (m >= M) continue;
    const int32_t rc = bit_offset(m, d.nm, d.cm);
    if (pairs) {
#pragma unroll
      for (int j = 0; j < WN; j += 2)
        if (cc[j] >= 0)
          *reinterpret_cast<float4*>(C + rc + cc[j]) = make_float4(accr[i][j], acci[i][j], accr[i][j + 1], acci[i][j + 1]);
    } else {
#pragma unroll
      for (int j = 0; j < WN; ++j)
        if (cc[j] >= 0) C[rc + cc[j]] = make_float2(accr[i][j], acci[i][j]);
    }
  }
}

template <int BN>
cudaError_t launch_bn(const float2* A, const float2* B, float2* C, const GemmDesc& d, int flags, cudaStream_t s) {
  constexpr int SMEM = 2 * BK * (BM + BN) * (int)sizeof(float2);
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(gemm_simt_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t M = int64_t(1) << d.nm, N = int64_t(1) << d.nn;
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)d.units);
  gemm_simt_kernel<BN><<<grid, NT, SMEM, s>>>(A, B, C, d, flags);
  return cudaGetLastError();
}

// Vector loads of 4 consecutive K values need the operand's two fastest
// indices to be its K bits 0 and 1 and every such quad to start on a 16-byte
// boundary: the base and the unit strides even (in complex elements), and the
// other strides even, which holds once bits 0 and 1 take strides 1 and 2.
bool quad_ok(const float2* base, int nk, const int32_t* kst, int64_t lo, int64_t hi) {
  return nk >= 2 && kst[0] == 1 && kst[1] == 2 && (reinterpret_cast<uintptr_t>(base) & 15) == 0 && (lo & 1) == 0 &&
         (hi & 1) == 0;
}

}  // namespace

cudaError_t launch_gemm_simt(const float2* A, const float2* B, float2* C, const GemmDesc& d, cudaStream_t s) {
  int flags = 0;
  if (quad_ok(A, d.nk, d.ak, d.a_lo, d.a_hi)) flags |= 1;
  if (quad_ok(B, d.nk, d.bk, d.b_lo, d.b_hi)) flags |= 2;
  // column bit 0 with C stride 1: columns 2j, 2j + 1 are adjacent and the
  // pair starts on an even element (every other stride of C is even)
  if (d.nn >= 1 && d.cn[0] == 1 && (reinterpret_cast<uintptr_t>(C) & 15) == 0 && (d.c_lo & 1) == 0 &&
      (d.c_hi & 1) == 0)
    flags |= 4;
  if (d.nn >= 7) return launch_bn<128>(A, B, C, d, flags, s);
  return launch_bn<64>(A, B, C, d, flags, s);
}

}  // namespace tn
