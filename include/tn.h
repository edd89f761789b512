/*
 * tn.h -- C ABI of the GB300 random-circuit tensor-network library.
 *
 * The library computes output amplitudes <x|U|0...0> of a random quantum
 * circuit U by contracting its tensor network (paper: Sec. "Existing Efforts
 * on Simulation of RQCs", tensor approach), sliced into 2^S independent
 * sub-networks whose results are summed (Sec. "A PEPS-based Simulation Method
 * with an Optimized Slicing Strategy"), with a batch of 2^k amplitudes per
 * contraction obtained by leaving k output qubits open (same section, "open
 * batch").  Each slice runs a planned chain of pairwise contractions, each an
 * index permutation fused into a complex GEMM (Sec. "Tensor Contraction Using
 * Fused Permutation and Multiplication"), in one of several precisions (Sec.
 * "A Mixed-Precision Computation Method via Adaptive Precision Scaling").
 *
 * Conventions used throughout:
 *  - Qubit q of an R x C grid is (r, c) with q = r*C + c.
 *  - Bitstrings are packed little-endian in ceil(n/64) uint64 words per
 *    bitstring: bit q of the word array is the value of qubit q.
 *  - Amplitude batch: output index j of a bitstring sets open qubit
 *    open_qubits[t] to bit t of j; the bitstring's own bits for open qubits
 *    are ignored.
 *  - Complex numbers are interleaved (re, im).  Amplitude outputs are
 *    complex128 (the cross-slice sum is FP64); device tensors are complex64.
 *  - Tensor indices all have dimension 2.  A rank-r tensor with index labels
 *    (l_0, ..., l_{r-1}) is stored row-major: element offset
 *    sum_t x_t * 2^(r-1-t), so l_0 is the slowest index.
 *
 * Ownership and errors: every function returns a tn_status (TN_OK = 0).  On
 * error a message describing the failure is available from tn_last_error()
 * (thread-local, valid until the next call on the same thread), and output
 * arguments are left untouched.  Handles are created and destroyed by the
 * library; arrays passed in are owned by the caller and only read during the
 * call.  All pointer and size arguments are validated on the host before any
 * device work is queued.  The tn_free_* functions accept NULL.
 */
#ifndef TN_H
#define TN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TN_OK = 0,
  TN_EINVAL = 1,      /* invalid argument (null pointer, bad size, bad label) */
  TN_ENOMEM = 2,      /* host allocation failed */
  TN_EHBM = 3,        /* device memory needed exceeds what is free */
  TN_ECUDA = 4,       /* a CUDA runtime call or kernel launch failed */
  TN_ETIMEOUT = 5,    /* a bounded device or host wait expired */
  TN_ETOOBIG = 6,     /* the plan's cost exceeds the caller's cap */
  TN_EOVERFLOW = 7,   /* a scaled low-precision slice over/underflowed and the policy forbids recompute */
  TN_ENOTREADY = 8,   /* a serving request has not completed yet */
  TN_ENODEVICE = 9,   /* no usable sm_103 device */
  TN_EINTERNAL = 10   /* unexpected host-side failure inside the library; the message names it */
} tn_status;

/* Human-readable description of the last error on this thread. */
const char* tn_last_error(void);
/* Library version string, e.g. "gb300-rqc-tn 0.1". */
const char* tn_version(void);

/* ------------------------------------------------------------------ */
/* Circuits (paper: Sec. "General Background of RQC")                  */
/* ------------------------------------------------------------------ */

enum {
  TN_GATE_SQRTX = 0, /* (1/sqrt2)[[1,-i],[-i,1]] */
  TN_GATE_SQRTY = 1, /* (1/sqrt2)[[1,-1],[1,1]] */
  TN_GATE_SQRTW = 2, /* (1/sqrt2)[[1,-e^{i pi/4}],[e^{-i pi/4},1]] */
  TN_GATE_FSIM = 3,  /* fSim(theta, phi), basis index 2*x_q0 + x_q1 */
  TN_GATE_MAT1 = 4,  /* arbitrary 2x2 in mat[0..7] */
  TN_GATE_MAT2 = 5   /* arbitrary 4x4 in mat[0..31], basis index 2*x_q0 + x_q1 */
};

/* One gate.  q1 = -1 for one-qubit gates; two-qubit gates need q0 != q1.
 * mat holds a row-major complex matrix as (re, im) pairs for MAT1/MAT2 and is
 * filled by the library for the named kinds when read back. */
typedef struct {
  int32_t kind;
  int32_t q0;
  int32_t q1;
  int32_t reserved;
  double theta;
  double phi;
  double mat[32];
} tn_gate;

typedef struct tn_circuit_s tn_circuit;

/* Seeded random circuit on a rows x cols grid with depth (1+depth+1): one
 * layer of one-qubit gates, then `depth` cycles of {fSim(pi/2, pi/6) layer on
 * coupler pattern A,B,C,D (cycle c uses pattern c mod 4), one-qubit layer}.
 * Patterns: A horizontal (r,c)-(r,c+1) c even; B horizontal c odd; C vertical
 * (r,c)-(r+1,c) r even; D vertical r odd.  One-qubit kinds are drawn from
 * {sqrtX, sqrtY, sqrtW} with SplitMix64(seed), uniform over k options via
 * ((x >> 32) * k) >> 32; after the first layer a qubit never repeats its
 * previous kind.  rows, cols >= 1, rows*cols <= 64, 0 <= depth <= 4096. */
tn_status tn_random_circuit(int32_t rows, int32_t cols, int32_t depth, uint64_t seed, tn_circuit** out);
/* Circuit from an explicit gate list (num_qubits <= 64). */
tn_status tn_circuit_from_gates(int32_t num_qubits, int64_t num_gates, const tn_gate* gates, tn_circuit** out);
tn_status tn_circuit_info(const tn_circuit* c, int32_t* num_qubits, int64_t* num_gates);
/* Copies the gate list into out[0 .. num_gates-1]. */
tn_status tn_circuit_gates(const tn_circuit* c, tn_gate* out, int64_t capacity);
void tn_free_circuit(tn_circuit* c);

/* ------------------------------------------------------------------ */
/* Tensor network (paper: Sec. "Existing Efforts on Simulation of RQCs") */
/* ------------------------------------------------------------------ */

typedef struct tn_network_s tn_network;

typedef struct {
  int32_t num_qubits;
  int32_t num_open;
  int32_t num_leaves;      /* tensors after simplification */
  int32_t num_labels;      /* distinct wire-segment indices in the leaves */
  int32_t max_leaf_rank;   /* including closed-output indices */
  int32_t num_closed;      /* closed output indices (fixed per bitstring) */
} tn_network_info;

/* Builds the network of <x|U|0^n> with the listed qubits left open (their
 * order defines the amplitude-batch index, see above).  Inputs |0> are
 * rank-1, one-qubit gates rank-2, two-qubit gates rank-4 tensors; each closed
 * output wire becomes a "fixed" index whose value is the bitstring bit at
 * contraction time.  Tensors of rank <= 2 (not counting fixed indices) are
 * absorbed into a neighbour (FP64 on the host).  open_qubits may be NULL when
 * num_open == 0; entries must be distinct and in [0, n). */
tn_status tn_build_network(const tn_circuit* c, const int32_t* open_qubits, int32_t num_open, tn_network** out);
/* Options of tn_build_network_ex. */
enum {
  /* Diagonal decomposition (Sec. "A PEPS-based Simulation Method with an
   * Optimized Slicing Strategy": diagonal gates turn their wire indices into
   * hyperedges).  Every two-qubit gate that is a wire swap times a diagonal
   * (fSim(pi/2, phi) = SWAP diag(1, -i, -i, e^{-i phi}); checked on the
   * matrix to 1e-12) gets no tensor: the swap renames the wires, and the
   * diagonal's two operator-Schmidt factors (bond index of dimension 2, named
   * (q, t) = (-1 - g, 0) for gate g) are merged into the tensors that produced
   * the two input wires, so every index still has two holders.  Raw tensor
   * ids of the factors (tn_plan_tree): num_gates + n + 2 g (the copy of wire
   * x_a into the bond) and num_gates + n + 2 g + 1 (D(bond, x_b)). */
  TN_NET_SPLIT_DIAGONAL = 1
};
/* tn_build_network with options (a bitwise OR of TN_NET_*; TN_EINVAL for
 * unknown bits). */
tn_status tn_build_network_ex(const tn_circuit* c, const int32_t* open_qubits, int32_t num_open, int32_t flags,
                              tn_network** out);
tn_status tn_network_get_info(const tn_network* net, tn_network_info* info);
/* Wire-segment name of a label: qubit q after its t-th gate (t = 0 is the
 * input wire); (-1 - g, 0) for the bond of gate g's split diagonal.
 * pairs_out receives 2*num_labels int32 (q, t). */
tn_status tn_network_label_wires(const tn_network* net, int32_t* pairs_out, int64_t capacity_pairs);
void tn_free_network(tn_network* net);

/* ------------------------------------------------------------------ */
/* Planning (paper: Secs. "A PEPS-based Simulation Method ..." and      */
/* "Searching for Better Contraction Paths with a Reduced Complexity")  */
/* ------------------------------------------------------------------ */

typedef struct tn_plan_s tn_plan_t;  /* opaque plan handle */

typedef struct {
  int32_t num_sliced;            /* exact number of sliced indices S; -1 = as few as the width cap needs */
  int32_t max_log2_intermediate; /* per-slice width cap (log2 elements); 0 = no cap */
  int32_t search_trials;         /* order-search restarts; 0 = default (128) */
  int32_t bitstrings_hint;       /* bitstrings expected per call: the search weighs the steps that
                                    depend on the bitstring (run once per bitstring and slice) by it
                                    against the slice-only ones (run once per slice); 0 = 1 */
  uint64_t seed;                 /* search seed; equal inputs + seed give byte-identical plans */
  double max_log2_cmac;          /* cost cap on total complex MACs (log2); 0 = none -> TN_ETOOBIG when exceeded */
  int32_t order_generator;       /* 0: randomized greedy + graph bisection (default); 1: PEPS-style
                                    lattice sweep (each grid column merged in time order, then the
                                    columns absorbed from one side; trials cycle through the four
                                    sweep directions), Sec. "A PEPS-based Simulation Method ..." */
  int32_t cap_aware_rewrites;    /* subtree rewrites after slicing (exact reordering of small
                                    subtrees) under a width cap: 0 = unconstrained, and the search
                                    is repeated with constrained rewrites only when no plan met the
                                    cap; 1 = always constrained (no rewrite builds an intermediate
                                    wider than the cap: often far cheaper plans under tight caps) */
} tn_plan_opts;

typedef struct {
  int32_t num_qubits;
  int32_t num_open;
  int32_t num_sliced;
  int32_t num_steps;
  int32_t num_leaves;
  int32_t max_log2_intermediate; /* largest per-slice tensor (log2 elements) */
  int64_t num_slices;            /* slice ids a call can address: 2^num_sliced, at most 2^62 (higher
                                    sliced indices then stay at 0) */
  double cmac_per_slice;         /* counted complex multiply-adds of one slice */
  double flops_per_slice;        /* 8 real flops per complex MAC (counted, not issued) */
  double log2_cmac_total;        /* log2(cmac_per_slice * num_slices) */
  int64_t footprint_bytes_per_unit; /* peak live complex64 bytes of one slice */
  uint64_t hash;                 /* FNV-1a 64 of the serialized plan */
  int32_t num_dense_steps;       /* steps routed to the tensor-core GEMM */
  int32_t num_vector_steps;      /* steps routed to the bandwidth kernel */
} tn_plan_info;

tn_status tn_plan(const tn_network* net, const tn_plan_opts* opts, tn_plan_t** out);
tn_status tn_plan_get_info(const tn_plan_t* p, tn_plan_info* info);
/* The sliced indices as (q, t) wire segments: sliced index j takes bit j of
 * the slice id.  pairs_out receives 2*num_sliced int32. */
tn_status tn_plan_sliced_wires(const tn_plan_t* p, int32_t* pairs_out, int64_t capacity_pairs);
/* Serialized plan bytes; call with buf = NULL to get the length. */
tn_status tn_plan_serialize(const tn_plan_t* p, uint8_t* buf, size_t capacity, size_t* len);
/* Contraction tree for replay: leaf_raw receives, per leaf, the raw tensor ids
 * it merges (-1 terminated lists, raw id g < num_gates = gate g, num_gates + q =
 * input vector of qubit q); tree receives 2*(num_leaves-1) SSA ids (leaves
 * 0..L-1, step i result L+i).  Sizes via tn_plan_get_info. */
tn_status tn_plan_tree(const tn_plan_t* p, int32_t* leaf_raw, int64_t leaf_raw_capacity, int32_t* tree, int64_t tree_capacity);

/* Where each tensor of a slice's contraction lives in device memory (the
 * planner's layout: a leaf store, an invariant store, and per-slice and
 * per-(bitstring, slice) arenas reused by liveness). */
typedef struct {
  int32_t phase;        /* 0: leaf store (a leaf) or invariant store (a step output);
                           1: slice arena (slice-only tensors); 2: pair arena (per bitstring and slice) */
  int32_t producer;     /* step writing the tensor; -1 for a leaf */
  int32_t consumer;     /* step reading it; -1 for the root */
  int32_t log2_elems;   /* complex64 elements as contracted (fixed indices removed), log2 */
  int64_t offset;       /* element offset in the memory named by phase (per slice / per unit for 1, 2) */
  int64_t store_offset; /* a leaf: element offset of the whole leaf in the leaf store; -1 for a step output */
  int32_t store_log2;   /* a leaf: log2 elements of the whole leaf (fixed indices included); -1 otherwise */
  int32_t step_class;   /* a step output: the planned class of its step: 0 dense (a GEMM: on the tensor
                           cores in a tensor-core precision when M >= 128, N >= 16 and K >= 8, else FP32),
                           1 vector-like (streaming kernels); -1 for a leaf */
  int32_t log2_m, log2_n, log2_k; /* a step output: its step's GEMM shape (M rows of A, N columns of B,
                                     K contracted); -1 for a leaf */
  int32_t reserved;
} tn_tensor_layout;

/* Fills out[x] for every SSA tensor x (leaves 0..L-1, step i's output L+i;
 * capacity >= num_leaves + num_steps) and arena_elems[0..3] with the sizes in
 * complex64 elements of the leaf store, the invariant store, the slice arena
 * (per slice) and the pair arena (per bitstring and slice). */
tn_status tn_plan_layout(const tn_plan_t* p, tn_tensor_layout* out, int64_t capacity, int64_t* arena_elems);
void tn_free_plan(tn_plan_t* p);

/* ------------------------------------------------------------------ */
/* Contraction (the hot path)                                          */
/* ------------------------------------------------------------------ */

enum {
  TN_PREC_C64 = 0,          /* complex64 storage, FP32 products and sums (SIMT FFMA) */
  TN_PREC_SPLIT_BF16 = 1,   /* complex64 storage; GEMMs as bf16 hi+lo split on tcgen05, FP32 accumulate */
  TN_PREC_SPLIT_FP16 = 2,   /* as above with fp16 hi+lo and a per-tensor power-of-two scale */
  TN_PREC_SCALED_FP16 = 3,  /* complex fp16 storage with per-tensor power-of-two scale, FP32 accumulate */
  TN_PREC_SCALED_BF16 = 4   /* complex bf16 storage with per-tensor power-of-two scale, FP32 accumulate */
};

typedef struct {
  void* stream;             /* cudaStream_t to run on; NULL = the legacy default stream */
  int32_t precision;        /* TN_PREC_* */
  int32_t device_io;        /* 0: bitstrings/out are host memory; 1: device memory */
  int64_t slice_begin;      /* first slice id of the summed range */
  int64_t slice_count;      /* number of slices summed; -1 = all from slice_begin */
  int32_t units_per_group;  /* slices contracted together per launch; 0 = auto */
  int32_t overflow_policy;  /* scaled modes: 0 = recompute a flagged slice in complex64, 1 = discard it (counted) */
  int32_t use_graph;        /* 1 = capture each group's launch sequence once per geometry as a CUDA graph and
                               replay it (needs a non-NULL stream; not with profile or test_flag_every) */
  int32_t profile;          /* 1 = bracket every kernel launch with CUDA events and fill the per-class figures */
  int32_t test_flag_every;  /* scaled modes, testing: > 0 flags every slice whose id is a multiple of it, so the
                               recompute / discard paths run without a real under/overflow; 0 = off */
  int32_t autotune;         /* 1 = time the tensor-core tile choices of every step on the first group of this
                               precision and keep the fastest (cached per plan; also in the file named by the
                               environment variable TN_AUTOTUNE_CACHE when it is set) */
  int32_t handover;         /* tensor-core precisions: 0 = default, 1 = a step feeding a tensor-core step writes
                               its output directly as 16-bit operand planes, 2 = it writes complex64 and the
                               consumer splits it (exact per-tensor scale) */
  int32_t reserved3;
  const int8_t* step_precision; /* NULL, or host array of one entry per plan step (num_steps of
                               tn_plan_get_info): TN_PREC_* for that step, -1 = `precision`.  Steps
                               that depend on neither slice nor bitstring always run in complex64.
                               Per-step precision (Sec. "A Mixed-Precision Computation Method via
                               Adaptive Precision Scaling": the precision-sensitive parts keep the
                               accurate format); tn_precision_analysis fills one.  Disables use_graph */
} tn_exec_opts;

/* Per-step precision from a pre-analysis (Sec. "A Mixed-Precision Computation
 * Method via Adaptive Precision Scaling": a pre-analysis on a few paths finds
 * the precision-sensitive parts, which keep the accurate format).  On a probe
 * -- the nb host bitstrings summed over slices [0, probe_slices) -- it
 * contracts the complex64 reference, then each candidate step (every step
 * after the plan-invariant phase whose GEMM fits the tensor cores) in
 * fast_precision with the other candidates in accurate_precision, orders the
 * candidates by the error each brings in, and keeps accurate the fewest most
 * sensitive steps whose mixed assignment meets target_rel_err (relative L2
 * against the reference) on the probe.  step_precision (num_steps entries,
 * caller-owned) receives the assignment for tn_exec_opts.step_precision:
 * fast_precision or accurate_precision on candidates, -1 elsewhere; when even
 * the all-accurate assignment misses the target every candidate is accurate
 * and rep->err_mixed says by how much.  Precisions must be 16-bit tensor-core
 * ones (TN_PREC_SPLIT_BF16 .. TN_PREC_SCALED_BF16); 1 <= nb <= 4096;
 * TN_EINVAL otherwise, before any work.  Synchronous; runs about
 * candidates + 2 log2(candidates) probe contractions on the current device. */
typedef struct {
  double err_fast;               /* probe error with every candidate fast */
  double err_accurate;           /* ... every candidate accurate */
  double err_mixed;              /* ... with the returned assignment */
  int32_t candidate_steps;
  int32_t accurate_steps;        /* candidates kept in accurate_precision */
  double accurate_flops_fraction;/* share of the candidates' counted work (per probe) that runs accurate */
  int32_t accurate_slice_only_steps; /* of the accurate steps, those that depend on the slice but not on the
                                        bitstring (the steps nearest the sliced indices) */
  int32_t probe_runs;            /* contractions the analysis ran */
} tn_precision_report;
tn_status tn_precision_analysis(tn_plan_t* p, const uint64_t* bitstrings, int64_t nb, int64_t probe_slices,
                                int32_t fast_precision, int32_t accurate_precision, double target_rel_err,
                                int8_t* step_precision, tn_precision_report* rep);

/* Kernel classes of the per-class report figures: FP32 GEMM, bandwidth-bound
 * streaming and reduction kernels, tensor-core GEMMs, operand split passes. */
enum { TN_KCLASS_GEMM_SIMT = 0, TN_KCLASS_VECTOR = 1, TN_KCLASS_GEMM_TC = 2, TN_KCLASS_SPLIT = 3 };

typedef struct {
  double device_ms;          /* device time of the call (CUDA events on the call's stream) */
  double flops;              /* counted flops of the work done (8 per complex MAC; shared work counted once) */
  double flops_equivalent;   /* counted flops of the same result without sharing slice-only work across bitstrings */
  int64_t units;             /* (bitstring, slice) units summed */
  int64_t kernel_launches;   /* kernels launched by the call */
  int64_t flagged_units;     /* scaled-mode units flagged for over/underflow */
  int64_t discarded_units;   /* flagged units dropped under overflow_policy = 1 */
  double class_ms[4];        /* profile = 1: summed launch durations per kernel class (TN_KCLASS_*) */
  int64_t class_launches[4];
  double class_flops[4];     /* counted flops of those launches */
  double class_bytes[4];     /* algorithmic bytes: each distinct operand read once, each output written once */
} tn_report;

/* Sums, over the slice range, the contraction of every bitstring's network:
 *   out[b*2^k + j] = sum_{s in range} C_{b,s}[j]   (complex128, (re, im))
 * bitstrings: nb * ceil(n/64) uint64 words; out: nb * 2^k complex128, with
 * nb * 2^k <= 2^40 (TN_EINVAL above).  Both
 * live on the host (device_io = 0) or the device (device_io = 1).  The call
 * is synchronous for host I/O; for device I/O it returns once work is queued
 * on opts->stream, except that the scaled precisions (their filter reads the
 * count of flagged units) and a non-NULL report wait for the device.  report
 * may be NULL. */
tn_status tn_contract_amplitudes(tn_plan_t* p, const uint64_t* bitstrings, int64_t nb, double* out,
                                 const tn_exec_opts* opts, tn_report* report);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of amplitude requests (the paper treats  */
/* slices as independent sub-tasks, Sec. "A Customized Parallelization  */
/* Scheme"; here one GPU interleaves the slices of many requests)        */
/* ------------------------------------------------------------------ */

typedef struct tn_server_s tn_server;

typedef struct {
  int32_t max_inflight;          /* requests contracted concurrently, one CUDA stream each; 0 = 4 (max 64) */
  int32_t slices_per_quantum;    /* slices of one request queued per scheduling turn; 0 = 64 */
  int32_t precision;             /* default TN_PREC_* of requests that ask for -1 */
  int32_t plan_trials;           /* order-search restarts per new circuit; 0 = 16 */
  int64_t hbm_budget_bytes;      /* device memory of the server; 0 = 60% of the free memory.  One
                                    eighth holds the stems of recent circuits, the rest bounds the
                                    estimated footprint of the admitted requests */
  double max_log2_cmac;          /* cost cap (log2 complex MACs a request is served, per
                                    bitstring); 0 = 48 */
  int32_t max_log2_intermediate; /* per-slice width cap when planning; 0 = 27 */
  int32_t planner_threads;       /* host threads planning new circuits concurrently; 0 = 4 (max 32) */
  int32_t over_cap_policy;       /* a request whose full plan costs more than the cap: 0 = fail it with
                                    TN_ETOOBIG; 1 = serve it at partial fidelity, from the largest
                                    leading range of slices that fits the cap (Sec. "A Mixed-Precision
                                    Computation Method via Adaptive Precision Scaling": a fraction f of
                                    the slices gives fidelity about f; tn_request_stats.slice_fraction
                                    reports f), TN_ETOOBIG only when one slice exceeds the cap */
  int32_t reserved;
} tn_server_opts;

/* One request: the amplitudes of nb bitstrings of the seeded random circuit
 * (tn_random_circuit(rows, cols, depth, seed)) with its last num_open qubits
 * open (2^num_open amplitudes per bitstring, batch index as in
 * tn_contract_amplitudes). */
typedef struct {
  int32_t rows, cols, depth;
  int32_t num_open;              /* 0 .. 12 */
  uint64_t seed;
  int64_t nb;                    /* 1 .. 2^24 */
  const uint64_t* bitstrings;    /* host, nb * ceil(n/64) words; copied by tn_submit */
  int32_t precision;             /* TN_PREC_*; -1 = the server default */
  int32_t reserved;
  double fidelity;               /* (0, 1): serve only the first ceil(fidelity * 2^S) slices
                                    of the plan's 2^S (Sec. "A Mixed-Precision Computation Method
                                    via Adaptive Precision Scaling": a fraction f of the slices
                                    gives amplitudes of fidelity about f); 0 or 1 = all slices.
                                    The server's cost cap applies to the slices served */
} tn_request;

typedef struct {
  double submit_to_done_ms;      /* latency seen by the caller */
  double queue_ms;               /* submit -> admitted (planning and waiting for a slot / budget) */
  double device_ms;              /* admitted -> amplitudes back on the host */
  double flops;                  /* counted flops of the request */
  int64_t slices;
  int32_t status;                /* the request's tn_status */
  int32_t num_open;
  int64_t nb;
  uint64_t plan_hash;
  int32_t planned_here;          /* 1 = this request ran the planner (plan cache miss) */
  int32_t stem_reused;           /* 1 = the circuit's leaf tensors and invariant (phase-0)
                                    intermediates were already resident from an earlier request */
  double slice_fraction;         /* slices served / 2^S: the expected fidelity of the amplitudes */
  double gpu_begin_ms;           /* device time (CUDA events, ms after the server's creation) at which the
                                    request's first slice quantum was reached on its stream */
  double gpu_end_ms;             /* device time at which its last quantum had finished */
  int64_t quanta;                /* slice quanta it was served in (one per scheduler turn) */
  int64_t batched_requests;      /* requests served by the same contraction (1 = alone): requests for the
                                    same circuit, open qubits, precision and slices that wait for
                                    admission together are merged, their bitstrings units of the same
                                    launches (at most 256 bitstrings in all) */
} tn_request_stats;

/* Creates a server on the current CUDA device with planner threads and a
 * scheduler thread.  Requests are admitted in arrival order when an in-flight
 * slot is free and their estimated device footprint fits the budget; admitted
 * requests advance one quantum of slices per turn each, on their own streams.
 * Plans are cached per circuit (the 256 most recently used, shared by the
 * servers of a process), and each circuit's stem (its leaf tensors and
 * the intermediates that depend on neither bitstring nor slice) stays
 * resident on the device for later requests of the same circuit, within one
 * eighth of the budget, least recently used first out.
 * A request's amplitudes are bit-identical whatever runs beside it. */
tn_status tn_server_create(const tn_server_opts* opts, tn_server** out);
/* Queues a request (arguments validated here; TN_ETOOBIG for a cost above the
 * cap and TN_EHBM for a request that can never fit are reported by tn_wait). */
tn_status tn_submit(tn_server* s, const tn_request* req, int64_t* ticket);
tn_status tn_poll(tn_server* s, int64_t ticket, int32_t* done);
/* Waits (timeout_s <= 0: no limit) for a request, copies its nb * 2^num_open
 * complex128 amplitudes to out (capacity in complex values), fills stats
 * (may be NULL), releases the ticket and returns the request's status. */
tn_status tn_wait(tn_server* s, int64_t ticket, double* out, int64_t capacity, tn_request_stats* stats,
                  double timeout_s);
/* Stops the threads, waits for the device and frees everything. */
void tn_server_destroy(tn_server* s);

/* ------------------------------------------------------------------ */
/* One pairwise contraction (Sec. "Tensor Contraction Using Fused       */
/* Permutation and Multiplication")                                    */
/* ------------------------------------------------------------------ */

enum {
  TN_PAIR_AUTO = 0,      /* the executor's kernel choice for this shape */
  TN_PAIR_FUSED_SIMT = 1,/* fused permute-GEMM, FP32 FFMA */
  TN_PAIR_VECTOR = 2,    /* bandwidth kernel (small N*K) */
  TN_PAIR_FUSED_TC = 3,  /* tcgen05 GEMM fed by TMA from split operand planes (library-allocated scratch) */
  TN_PAIR_UNFUSED = 4,   /* permute A and B to GEMM order, GEMM, permute C (library-allocated scratch) */
  TN_PAIR_GATHER_TC = 5, /* tcgen05 GEMM gathering and splitting operand tiles in the main loop (no scratch) */
  TN_PAIR_REDUCE = 6     /* bandwidth kernel for M N <= 64 outputs and K >= 256 (warp-shuffle reduction over K) */
};

/* C[c_labels] = sum over labels shared by A and B of A[a_labels] * B[b_labels].
 * A, B, C: device complex64 tensors (rank <= 30 each, row-major as above).
 * Every label of C appears in exactly one of A, B; a label shared by A and B
 * must not appear in C; labels are distinct within a tensor.
 * precision selects the arithmetic of the tensor-core algorithms:
 * TN_PREC_SPLIT_BF16 (hi + lo split, no scaling), TN_PREC_SPLIT_FP16 (hi + lo
 * split of operands scaled by their exact maxima), TN_PREC_SCALED_FP16 and
 * TN_PREC_SCALED_BF16 (one 16-bit product per real product, operands scaled
 * by their exact maxima, Sec. "A Mixed-Precision Computation Method via
 * Adaptive Precision Scaling"); C is complex64 with the scales undone.  The
 * gathering tensor-core kernel runs split bf16 only; the other algorithms
 * compute in FP32 whatever the precision.  TN_PAIR_AUTO picks the TMA
 * tensor-core kernel for any 16-bit precision when the shape allows it.
 * Asynchronous on `stream`, except the tensor-core algorithms, which return
 * once the kernel has finished (they check its error word). */
tn_status tn_contract_pair(const void* A, const int32_t* a_labels, int32_t a_rank,
                           const void* B, const int32_t* b_labels, int32_t b_rank,
                           void* C, const int32_t* c_labels, int32_t c_rank,
                           int32_t precision, int32_t algo, void* stream);

/* Failure detection of the tensor-core pipelines (Sec. "A Customized
 * Parallelization Scheme" runs every sub-task to completion; the bound below
 * is this library's own guard against a pipeline that stops making progress,
 * the paper has none).  Every wait of a TMA-fed tensor-core kernel (the
 * kernels of TN_PAIR_FUSED_TC and of tn_contract_amplitudes' 16-bit
 * precisions) polls its barrier at most `polls` times; a wait that runs out
 * records an error code, the CTA stops issuing work, waits (with the default
 * bound) for the copies and MMAs it already issued, releases its shared
 * memory and TMEM and exits, and the host call returns TN_ETIMEOUT.
 * polls < 0 restores the default (2^24); 0 makes every pipeline wait give up
 * at once (used by the tests of the TN_ETIMEOUT path).  Applies to the
 * current device, for every later launch until changed; synchronous.
 * Returns TN_ECUDA if the device symbol cannot be written. */
tn_status tn_set_wait_limit(int64_t polls);

/* Allocation-free variant of tn_contract_pair's tensor-core path (the paper
 * has no counterpart: this serves callers that cannot let a library allocate
 * device memory -- a framework whose caching allocator already holds the free
 * HBM, a serving loop with a fixed memory budget or no allocator calls on its
 * request path, code next to a CUDA graph capture).
 * Same arguments and label rules as tn_contract_pair with algo =
 * TN_PAIR_FUSED_TC and precision = TN_PREC_SPLIT_BF16 (M >= 128, N >= 16,
 * K >= 8).  Scratch comes from one static device array of 64 MiB per GPU
 * (kept until the process exits): the split operand planes,
 * 8 * (M + N) * K bytes, must fit, else TN_EINVAL before any work.
 * The first call on a device (that device current) looks up the array's
 * address with cudaGetSymbolAddress; make it before any stream capture.  All
 * calls on a device share the array: calls whose work overlaps on the GPU
 * race and must be serialised by the caller.  No cudaMalloc, cudaFree or
 * allocating library call is made.  Returns after the contraction has finished
 * on `stream` (it reads back the kernel's error word). */
tn_status tn_contract_pair_noalloc(const void* A, const int32_t* a_labels, int32_t a_rank,
                                   const void* B, const int32_t* b_labels, int32_t b_rank,
                                   void* C, const int32_t* c_labels, int32_t c_rank, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TN_H */
