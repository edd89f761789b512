// Device-side descriptors and kernel launchers shared by the executor and the
// pairwise-contraction entry point.
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace tn {

constexpr int kMaxBits = 32;

// One pairwise contraction C[m, n] = sum_k A[m, k] B[k, n] with M = 2^nm,
// N = 2^nn, K = 2^nk, where every operand is addressed through per-bit
// element strides: the index permutation of each operand (paper: Sec. "Tensor
// Contraction Using Fused Permutation and Multiplication") is folded into the
// address arithmetic instead of being materialised.  Element (m, k) of A sits
// at sum_i bit_i(m) am[i] + sum_l bit_l(k) ak[l] (+ unit * a_unit), and
// likewise for B (k, n) and C (m, n).  Bits are numbered so that bit 0 is the
// operand's most contiguous index of that group.
//
// A launch covers `units` units; unit u splits into (u % units_lo, u / units_lo)
// and each operand's base moves by (u % units_lo) * x_lo + (u / units_lo) * x_hi
// elements, so an operand shared by some units (a slice-only tensor read by
// every bitstring of the slice, or an invariant one) simply has a zero stride.
struct GemmDesc {
  int nm, nn, nk;
  int units, units_lo;
  int tile_n, group_m;       // tensor-core tile width / raster group (0 = default; set by the autotuner)
  int persistent;            // tensor-core GEMM: 0 auto, 1 persistent CTAs (double-buffered accumulators), 2 one tile per CTA
  int64_t a_lo, a_hi, b_lo, b_hi, c_lo, c_hi;
  int32_t am[kMaxBits], cm[kMaxBits];
  int32_t bn[kMaxBits], cn[kMaxBits];
  int32_t ak[kMaxBits], bk[kMaxBits];
};

// Variant leaf: the sub-tensor of one unit is the full leaf with its fixed
// indices set to the unit's values (sliced index j <- bit j of the slice id;
// closed output qubit q <- bit q of the bitstring).
constexpr int kMaxLeafRank = 12;
struct LeafGather {
  int64_t store_off;         // full leaf in the leaf store
  int64_t dst_off;           // sub-tensor in the unit arena
  int32_t nkept, nfixed;
  int32_t kept_stride[kMaxLeafRank];   // full-leaf stride of each kept index, slowest first
  int32_t fixed_src[kMaxLeafRank];     // >= 0: slice bit j; <= -2: closed qubit (-src-2)
  int32_t fixed_stride[kMaxLeafRank];
};

// A group of units: `nslice` consecutive slice ids from slice0 for the
// bitstrings b0 .. b0+nb-1; unit u = (u % nslice) slice, (u / nslice) bitstring.
// The kernels read it from a device slot written by launch_set_group, so a
// captured launch sequence can be replayed for any group.
struct GroupInfo {
  int64_t slice0;
  int64_t b0;
  int32_t nslice;
  int32_t nb;                // 1 for slice-only launches
  int32_t words;             // uint64 words per bitstring
  int32_t units;             // nslice * nb
  const uint64_t* bits;      // bitstrings of the call (device)
  double2* acc;              // amplitude accumulator of the call (device)
};

// launchers (return cudaGetLastError())
cudaError_t launch_gemm_simt(const float2* A, const float2* B, float2* C, const GemmDesc& d, cudaStream_t s);
// tcgen05 fused permute-GEMM (complex64 in/out, 16-bit hi+lo split products,
// FP32 accumulation).  Operands are multiplied by a_scale / b_scale before the
// split and the result divided by their product (powers of two).  *err is set
// non-zero when a bounded wait expired.
bool tc_shape_ok(const GemmDesc& d);
cudaError_t launch_gemm_tc(const float2* A, const float2* B, float2* C, const GemmDesc& d, bool bf16, float a_scale,
                           float b_scale, int* err, cudaStream_t s);
// Operand preparation for the TMA-fed GEMM: rows = M (A) or N (B), each row a
// K run; element (r, k) at sum bit_i(r) row_st[i] + sum bit_l(k) k_st[l] of
// the source tensor number z, whose base is src + (z % nlo) * lo + (z / nlo) * hi.
// Output: per z four planes {re_hi, re_lo, im_hi, im_lo} of rows_pad x kp
// 16-bit values (kp = K >= 8; the GEMM's TMA copies read past a short K as zeros).
struct SplitDesc {
  int nrow, nk;
  int rows_pad, kp;
  int nlo;
  int kvec;  // 8 consecutive K values contiguous and 16-byte aligned: vector loads
  int64_t lo, hi;
  int32_t row_st[kMaxBits], k_st[kMaxBits];
};
// max_ready: maxbits already holds each operand tensor's largest |component|
// (recorded by its producer), so the maximum pass is skipped.
cudaError_t launch_split(const float2* src, uint16_t* dst, const SplitDesc& d, int nz, bool bf16, int np,
                         unsigned* maxbits, int* e_out, float* m_out, cudaStream_t s, bool max_ready = false);
// One GEMM operand stored as four K-major 16-bit planes {re_hi, re_lo, im_hi,
// im_lo}, each rows x kp; consecutive units are st_lo / st_hi bytes apart
// along the two unit dimensions (extent 1 = one tensor shared by all units).
struct PlaneOperand {
  const uint16_t* base;
  int np;                // 4 planes (re_hi, re_lo, im_hi, im_lo) or 2 (re, im)
  int64_t kp, rows;
  int64_t nlo, nhi;
  int64_t st_lo, st_hi;
};
// TMA-fed warp-specialized tcgen05 GEMM on plane operands.  With c_planes
// the epilogue writes C as planes (for a tensor-core consumer) instead of
// complex64.
int tma_tile_n(const GemmDesc& d);
// I/O of the scaled precisions; every pointer may be null (exponent 0, no
// tracking).  ea/ma, eb/mb: per distinct operand tensor, the exponent e of
// its stored values (stored = true * 2^-e) and their largest |component|.
// ec/mc: the same for a plane output (mc as float bits, atomicMax; cleared by
// the caller).  flag: per launch unit (or per low unit index when flag_by_lo)
// set when values turn non-finite or an operand maximum is below 2^-10.
struct ScaleIO {
  const int* ea;
  const float* ma;
  const int* eb;
  const float* mb;
  int* ec;
  unsigned* mc;
  int* flag;
  int flag_by_lo;
};
int64_t split_plane_elems(int nrow_bits, int nk_bits, int np);
// Polls of every pipeline wait of the TMA tensor-core kernels on the current
// device (negative: the default, 2^24).  A wait that runs out records an
// error code in the kernel's error word and the CTA winds down.
cudaError_t set_tc_wait_limit(long long polls);
cudaError_t launch_gemm_tma(const PlaneOperand& a, const PlaneOperand& b, float2* C, bool c_planes, const GemmDesc& d,
                            bool bf16, const ScaleIO& sio, int* err, cudaStream_t s);
// Split operand A (which_b = false) or B of d into `scratch` (returned planes).
// With `scaled`, each distinct tensor z is first reduced to its largest
// |component| (maxbits[z], cleared by the caller) and stored times 2^-e_z with
// e_z chosen so that this maximum lands in [2^13, 2^14); e_out / m_out receive
// e_z and the stored maximum.
int64_t split_scratch_elems(const GemmDesc& d, bool which_b, int np);
cudaError_t split_operand(const float2* src, const GemmDesc& d, bool which_b, bool bf16, int np, bool scaled,
                          unsigned* maxbits, int* e_out, float* m_out, uint16_t* scratch, PlaneOperand& out,
                          cudaStream_t s, bool max_ready = false);
// Plane operand of a tensor a producer epilogue already wrote as np planes
// (layout [rows][K], K >= 8); false when the step's view does not match.
bool planes_in_place(const float2* base, const GemmDesc& d, bool which_b, int np, PlaneOperand& out);
// Split both operands of d into `scratch` (>= tc2_scratch_elems(d) 16-bit
// values) and run the TMA GEMM.
int64_t tc2_scratch_elems(const GemmDesc& d);
cudaError_t run_gemm_tc2(const float2* A, const float2* B, float2* C, const GemmDesc& d, bool bf16, uint16_t* scratch,
                         int* err, cudaStream_t s);
// Same with both operands scaled by their exact maxima (one power-of-two
// exponent each) and split into np planes (4: split fp16/bf16, 2: scaled
// single products); C is written in complex64 with the exponents applied.
// aux: 24 bytes of device memory (maxima, exponents, stored maxima).
cudaError_t run_gemm_tc2_scaled(const float2* A, const float2* B, float2* C, const GemmDesc& d, bool bf16, int np,
                                uint16_t* scratch, void* aux, int* err, cudaStream_t s);
// Vector-like steps: N <= 16 and K <= 16, N <= 8 and K <= 128, N <= 256 and
// K <= 4, or N = 32 and K = 8 (k_vector.cu).
bool vector_shape_ok(const GemmDesc& d);
// Shapes the tensor cores could take that run faster on the streaming kernel.
bool stream_preferred(const GemmDesc& d);
// Output of a streaming step.  mode 0: complex64 C; 2: four 16-bit planes
// {re_hi, re_lo, im_hi, im_lo} (bf16 or fp16, each `plane` elements, at C's
// element offsets: a tensor-core consumer's operand, unscaled).  maxbits (may
// be null): per launch unit, the largest |component| computed, as float bits
// by atomicMax (cleared by the caller).
struct VecOut {
  unsigned* maxbits;
  int mode;
  int bf16;
  int64_t plane;
};
cudaError_t launch_vector(const float2* A, const float2* B, float2* C, const GemmDesc& d, cudaStream_t s,
                          const VecOut& out = VecOut{});
// Few outputs (M N <= 64), long contracted index (K >= 256): one CTA per
// unit, K spread over the threads, warp-shuffle reduction (k_reduce.cu).
bool reduce_shape_ok(const GemmDesc& d);
cudaError_t launch_reduce(const float2* A, const float2* B, float2* C, const GemmDesc& d, cudaStream_t s);
cudaError_t launch_set_group(GroupInfo* slot, const GroupInfo& g, cudaStream_t s);
// grid covers `units` units (the slot's count may be lower for a partial group)
cudaError_t launch_gather(const float2* store, float2* arena, int64_t arena_stride, const LeafGather* descs,
                          int nleaves, const GroupInfo* slot, int units, cudaStream_t s);
// acc[b, j] += sum over the group's slices (in slice order) of root(b, s)[perm[j]],
// root(b, s) = root + s_local * r_lo + b_local * r_hi.
// Flagged units (flag_s per slice of the group, flag_u per unit; both may be
// null) are skipped and appended as (b << 32 | s) to `flagged` (capacity cap).
cudaError_t launch_accumulate(const float2* root, int64_t r_lo, int64_t r_hi, const int64_t* perm, int nperm,
                              const GroupInfo* slot, int nb_max, const int* flag_s, const int* flag_u,
                              int64_t* flagged, unsigned long long* nflagged, int cap, cudaStream_t s);
// dst (dense, element e) = src[sum_p bit_p(e) * st[p]]: bit p of e is dst's
// p-th fastest index, st[p] its element stride in src.
struct PermDesc {
  int rank;
  int32_t st[kMaxBits];
};
cudaError_t launch_permute(const float2* src, float2* dst, const PermDesc& p, int64_t units, int64_t src_unit,
                           int64_t dst_unit, cudaStream_t s);

struct Step;
// GEMM view (per-bit strides) of one pairwise step.
// m_by_output: number the M bits by the output's memory order (bandwidth
// kernel) instead of A's (GEMM kernels, whose A rows follow A's layout).
void make_gemm_desc(const std::vector<int>& la, const std::vector<int>& lb, const std::vector<int>& lc,
                    GemmDesc& d, bool m_by_output = false);

}  // namespace tn
