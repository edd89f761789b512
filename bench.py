"""Benchmark of the amplitude hot path (one JSON line on rank 0).

Workload (default): the 8x8 grid random circuit of depth 1+20+1 (circuit
seed 4), its network sliced so that no per-slice intermediate exceeds 2^26
complex elements, the first 4096 slices summed (a partial sum of fidelity
4096 / 2^S), the last ten qubits open: 1024 correlated amplitudes in FP16
hi+lo split precision with the FP64 cross-slice sum.  One "step" contracts
every slice for the batch and sums them: the whole hot path (slice
selection, the pairwise permute-GEMM chain, the cross-slice sum).
`--workload 6x6` runs the 6x6 grid of depth 1+16+1 (seed 2), 10 sliced
indices (1024 slices), six open qubits, four batches of 64 amplitudes.

`value` is counted complex-flop throughput (8 real flops per complex
multiply-add of the work actually performed, work shared by the batches
counted once) with inputs resident in HBM; `amplitudes_per_s` beside it.
`e2e` repeats the step through the C ABI with host buffers (bitstrings in,
amplitudes out, copies inside the timed region).  `roofline` describes the
dominant kernel class from per-launch CUDA events during the timed steps;
`cpu_baseline` times the FP64 CPU oracle on one slice of one batch (median
of three runs).  `precision_modes` times the other precisions on the same
workload (plain complex64 on a leading range of slices), each with its error
against the FP64 oracle on a sampled slice; `workload_6x6` does the same for
the 6x6 configuration; `serving` runs a Poisson request stream through the
plain one-slice-at-a-time complex64 path and the batched server.

Modes:
  python bench.py [--gpus N --steps K --warmup W] [--workload 8x8|6x6] [--precision split_fp16|...]
  python bench.py --impl reference ...   # the CPU oracle as the reference arm
  python bench.py --micro [--shape m,n,k]  # pairwise contraction microbenchmark
  python bench.py --serve [--requests R]   # serving: batched mixed precision vs plain complex64
Under torchrun each rank runs its own batches (weak scaling, no collective on
the data path); rank 0 prints the max-over-ranks timing.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Contraction TFLOP/s & amplitudes/s at stated rel err vs FP64; p50/p99 latency"
# the two single-GPU amplitude workloads (grid, depth, circuit seed, sliced
# indices (-1: as many as the width cap needs), per-slice width cap (0: none),
# open qubits, bitstring batches, bitstring seed, planner trials, slices summed
# (-1: all))
WORKLOADS = {
    "8x8": dict(rows=8, cols=8, depth=20, cseed=4, nsliced=-1, width_cap=26, nopen=10, nbatch=1, bseed=4,
                trials=16, slices=4096,
                text="8x8 grid, depth 1+20+1, fSim(pi/2,pi/6); per-slice width <= 2^26; first 4096 slices; "
                     "10 open qubits; 1 batch x 1024 correlated amplitudes"),
    "6x6": dict(rows=6, cols=6, depth=16, cseed=2, nsliced=10, width_cap=0, nopen=6, nbatch=4, bseed=2,
                trials=64, slices=-1,
                text="6x6 grid, depth 1+16+1, fSim(pi/2,pi/6); 10 sliced indices (1024 slices); 6 open qubits; "
                     "4 batches x 64 amplitudes"),
}
ROWS = COLS = DEPTH = CSEED = NSLICED = WIDTH_CAP = NOPEN = NBATCH = BSEED = PLAN_TRIALS = SLICE_LIMIT = None
WORKLOAD = None
PLAN_SEED, PLAN_HINT, PLAN_CAP_AWARE = 1, 0, 0
PLAN_SEEDS = 1  # planner seeds searched (PLAN_SEED, PLAN_SEED + 1, ...): the cheapest plan per slice is kept


def use_workload(name):
    global ROWS, COLS, DEPTH, CSEED, NSLICED, WIDTH_CAP, NOPEN, NBATCH, BSEED, PLAN_TRIALS, SLICE_LIMIT, WORKLOAD
    w = WORKLOADS[name]
    ROWS, COLS, DEPTH, CSEED = w["rows"], w["cols"], w["depth"], w["cseed"]
    NSLICED, WIDTH_CAP, NOPEN, NBATCH, BSEED = w["nsliced"], w["width_cap"], w["nopen"], w["nbatch"], w["bseed"]
    PLAN_TRIALS, SLICE_LIMIT, WORKLOAD = w["trials"], w["slices"], w["text"]


use_workload("8x8")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), \
            d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 1900.0, 1700.0, 2070.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                f = [x.strip() for x in out.stdout.strip().split(",")]
                if len(f) == 7:
                    self.samples.append(f)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if "Active" in s[3 + i]
                          and "Not" not in s[3 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def make_workload(T, rank):
    c = T.random_circuit(ROWS, COLS, DEPTH, CSEED)
    n = ROWS * COLS
    open_q = list(range(n - NOPEN, n))
    net = T.build_network(c, open_q)
    t0 = time.time()
    p = best_plan_of_seeds(T, net, range(PLAN_SEED, PLAN_SEED + PLAN_SEEDS))
    plan_s = time.time() - t0
    import tn_inputs as I
    words = I.bitstrings(n, NBATCH, BSEED + 1000 * rank)
    return c, net, p, words, open_q, plan_s


def best_plan_of_seeds(T, net, seeds):
    """The workload's plan from each planner seed; kept: the lowest work per
    slice (the benchmark sums a fixed number of slices), then fewer sliced
    indices.  Host planning only."""
    best, key = None, None
    for seed in seeds:
        p = T.plan(net, num_sliced=NSLICED, max_log2_intermediate=WIDTH_CAP, search_trials=PLAN_TRIALS, seed=seed,
                   bitstrings_hint=PLAN_HINT, cap_aware_rewrites=PLAN_CAP_AWARE)
        info = p.info()
        k = (info["cmac_per_slice"], info["num_sliced"])
        if best is None or k < key:
            best, key = p, k
    return best


def cpu_oracle_sample(p, words, open_q, slice_id=0):
    """FP64 oracle on one slice of one bitstring batch; returns (value, seconds, cmac)."""
    import tn_inputs as I
    from oracle import circuit as OC
    from oracle.replay import contract_in_order, work_cmac
    n = ROWS * COLS
    gates = OC.random_circuit(ROWS, COLS, DEPTH, CSEED)
    bits = I.bits_of(words[0], n)
    wires = p.sliced_wires()
    fixed = {wires[j]: (slice_id >> j) & 1 for j in range(len(wires))}
    leaves, pairs = p.tree(len(gates), n)
    t0 = time.time()
    v = contract_in_order(gates, n, bits, open_q, leaves, pairs, fixed)
    dt = time.time() - t0
    cmac = work_cmac(gates, n, bits, open_q, leaves, pairs, fixed)
    return v, dt, cmac


def traffic_record(kernel_file, key):
    """Per-launch DRAM bytes of the dominant kernel class for `key`
    ("<workload>/<precision>") from the committed ncu capture of the bench, if
    it was taken on the current source of the kernel file (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    src = os.path.join(ROOT, "paper_2110_14502_gb300", "csrc", kernel_file)
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    r = rec.get(kernel_file)
    if not r or r.get("source_sha") != h:
        return None
    return r.get(key)


MODES = ("split_fp16", "split_bf16", "scaled_fp16", "scaled_bf16", "c64")
DTYPE = {"split_bf16": "bf16x3", "split_fp16": "f16x3", "scaled_fp16": "f16", "scaled_bf16": "bf16", "c64": "f32"}
# plain complex64 runs on the FP32 CUDA cores: time it on a leading range of
# the slices (every slice of a plan does the same work)
C64_SLICE_FRACTION = {"8x8": 16, "6x6": 8}


def oracle_reference(p, words, open_q, runs=1):
    """FP64 oracle on slice 0 of batch 0: (values, [seconds per run], cmac)."""
    times = []
    for _ in range(runs):
        v, dt, cmac = cpu_oracle_sample(p, words, open_q, slice_id=0)
        times.append(dt)
    return v, times, cmac


def rel_err(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def time_mode(p, dwords, out, stream, mode, slices, frac, nout):
    """One warm-up and one timed call of `mode` on the first slices / frac
    slices (frac 1: the whole step); counted TFLOP/s and amplitudes/s of the
    whole step projected from the timed slice range."""
    import torch
    part = max(1, slices // frac)
    for rep_ in (False, True):
        with torch.cuda.stream(stream):
            _, r = p.contract_amplitudes(dwords, out=out, stream=stream, precision=mode, report=True,
                                         slice_count=part)
        torch.cuda.synchronize()
    ms_step = r["device_ms"] * slices / part
    e = {"tflops": round(r["flops"] / r["device_ms"] / 1e9, 2), "ms_per_step": round(ms_step, 1),
         "amplitudes_per_s": round(nout / (ms_step * 1e-3), 3), "flagged_units": r["flagged_units"]}
    if part < slices:
        e["slices_timed"] = part
        e["note"] = f"timed on slices 0..{part - 1} of {slices}; step time projected (equal work per slice)"
    return e


def mode_errors(p, words, ref, modes):
    out = {}
    for mode in modes:
        g1 = p.contract_amplitudes(words[:1], precision=mode, slice_begin=0, slice_count=1)[0]
        out[mode] = rel_err(g1, ref)
    return out


def run_ours(args):
    import torch
    import paper_2110_14502_gb300 as T

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        # replicas share nothing on the data path: the process group (gloo,
        # on the host) only carries the barriers and the max-over-ranks time
        import torch.distributed as dist
        dist.init_process_group("gloo")
    c, net, p, words, open_q, plan_s = make_workload(T, rank)
    info = p.info()
    k = info["num_open"]
    nout = NBATCH << k
    slices = info["num_slices"] if SLICE_LIMIT < 0 else min(SLICE_LIMIT, info["num_slices"])
    if args.slices > 0:
        slices = min(slices, args.slices)
    stream = torch.cuda.Stream()
    dwords = torch.from_numpy(words.astype(np.int64)).cuda()
    out = torch.empty(nout * 2, dtype=torch.float64, device="cuda")
    tune = 1 if args.autotune else 0

    def step(profile=False):
        with torch.cuda.stream(stream):
            _, rep = p.contract_amplitudes(dwords, out=out, stream=stream, precision=args.precision,
                                           profile=profile, report=True, slice_count=slices, autotune=tune)
        return rep

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    reps, times = [], []
    with Clocks(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            r = step(profile=True)
            reps.append(r)
            times.append(r["device_ms"])
        e1.record(stream)
        torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    flops = sum(r["flops"] for r in reps) * world
    flops_eq = sum(r["flops_equivalent"] for r in reps) * world
    amps = nout * args.steps * world
    value = flops / (total_ms * 1e-3) / 1e12
    launches = int(sum(r["kernel_launches"] for r in reps))  # every launch of the timed steps

    # roofline of the dominant kernel class over the timed steps
    hbm, bf16, bf16_sus, sm_max, src = peaks()
    cls_ms = [sum(r["class_ms"][i] for r in reps) for i in range(4)]
    cls_fl = [sum(r["class_flops"][i] for r in reps) for i in range(4)]
    cls_by = [sum(r["class_bytes"][i] for r in reps) for i in range(4)]
    cls_n = [sum(r["class_launches"][i] for r in reps) for i in range(4)]
    dom = int(np.argmax(cls_ms[:3]))
    kernel_file = {0: "k_simt.cu", 1: "k_vector.cu", 2: "k_tc2.cu"}[dom]
    tr = traffic_record(kernel_file, f"{args.workload}/{args.precision}")
    if dom == 2:
        achieved = cls_fl[dom] / (cls_ms[dom] * 1e-3) / 1e12
        # split precisions issue three 16-bit products per real product: the
        # peak of that arithmetic in counted flops is the bf16 peak / 3
        mult = 3 if args.precision.startswith("split") else 1
        peak = bf16_sus / mult
        roof = {"bound": "tensor", "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4),
                "peak_kind": f"bf16 dense sustained ({src}; fp16 runs at the same rate)" +
                             (" / 3 (three 16-bit MMAs per counted product)" if mult == 3 else ""),
                "issued_mma_tflops": round(mult * achieved, 2),
                "frac_of_bf16_peak_counted": round(achieved / bf16_sus, 4)}
    elif dom == 1:
        achieved = cls_by[dom] / (cls_ms[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "peak_kind": f"HBM copy ({src})"}
    else:
        achieved = cls_fl[dom] / (cls_ms[dom] * 1e-3) / 1e12
        fp32 = 152 * 128 * 2 * sm_max * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(fp32, 1), "unit": "TFLOP/s",
                "frac": round(achieved / fp32, 4), "peak_kind": "FP32 FFMA: 152 SMs x 128 lanes x 2 x max clock"}
    roof["kernel"] = {0: "gemm_simt_kernel", 1: "vector_kernel",
                      2: "gemm_tma_chunked" if args.precision.startswith("split")
                      else "gemm_tma_persistent / gemm_tma_kernel"}[dom]
    roof["launches_per_step"] = cls_n[dom] / args.steps
    roof["share_of_device_time"] = round(cls_ms[dom] / sum(cls_ms), 4) if sum(cls_ms) else None
    if cls_n[3]:
        roof["split_pass"] = {"ms_per_step": round(cls_ms[3] / args.steps, 2),
                              "gbs": round(cls_by[3] / (cls_ms[3] * 1e-3) / 1e9, 1),
                              "share_of_device_time": round(cls_ms[3] / sum(cls_ms), 4)}
    roof["algorithmic_bytes_per_launch"] = round(cls_by[dom] / cls_n[dom]) if cls_n[dom] else None
    roof["traffic"] = None if tr is None else tr["bytes_per_launch"]
    roof["traffic_note"] = None if tr is None else tr["note"]

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision],
        "data": "synthetic (seeded random circuit and bitstrings)",
        "config": {"workload": WORKLOAD, "precision": args.precision, "global_batch": amps // args.steps,
                   "slices": slices, "num_sliced": info["num_sliced"],
                   "fidelity_fraction_log2": round(float(np.log2(slices)) - info["num_sliced"], 3),
                   "plan_hash": hex(info["hash"]),
                   "cmac_per_slice_log2": round(float(np.log2(info["cmac_per_slice"])), 3),
                   "max_log2_intermediate": info["max_log2_intermediate"],
                   "l2": f"working set (2^{info['max_log2_intermediate']}-element complex64 intermediates per "
                         "slice, many slices per launch) larger than L2; no flush",
                   "parallelism": f"slices x bitstrings per GPU; {world} independent replica(s)"},
        "amplitudes_per_s": round(amps / (total_ms * 1e-3), 3),
        "flops_equivalent_tflops": round(flops_eq / (total_ms * 1e-3) / 1e12, 3),
        "p50_ms": round(float(np.percentile(times, 50)), 3), "p99_ms": round(float(np.percentile(times, 99)), 3),
        "plan_s": round(plan_s, 3),
        "gpu_launches": launches, "gpu_launches_per_step": launches // args.steps,
        "roofline": roof,
        "clocks": clk.summary(),
    }
    if not args.no_e2e:
        # e2e: pinned host buffers through the C ABI, copies inside the timed region
        words_h = torch.from_numpy(words.view(np.int64)).pin_memory().numpy().view(np.uint64)
        amps_h = torch.empty(nout, dtype=torch.complex128).pin_memory().numpy().reshape(NBATCH, 1 << k)
        e2e_times = []
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.time()
            p.contract_amplitudes(words_h, precision=args.precision, slice_count=slices, out=amps_h,
                                  autotune=tune)
            e2e_times.append(time.time() - t0)
        e2e_s = sum(e2e_times)
        e2e_flops = reps[0]["flops"] * len(e2e_times)
        line["e2e"] = {"value": round(e2e_flops / e2e_s / 1e12, 3), "unit": "TFLOP/s",
                       "amplitudes_per_s": round(nout * len(e2e_times) / e2e_s, 3),
                       "h2d_bytes_per_step": int(words_h.nbytes), "d2h_bytes_per_step": int(amps_h.nbytes),
                       "host_buffers": "pinned"}
    ref = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ref, dts, cmac = oracle_reference(p, words, open_q, runs=3)
        med, best = statistics.median(dts), min(dts)
        line["cpu_baseline"] = {"value": round(8 * cmac / med / 1e12, 6), "unit": "TFLOP/s",
                                "best_of_3": round(8 * cmac / best / 1e12, 6),
                                "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                                "sample": f"slice 0 of batch 0 ({1 << NOPEN} amplitudes, one slice of {slices}), "
                                          f"FP64 NumPy contraction in the plan's order; median of 3 runs "
                                          f"({', '.join(f'{x:.1f}' for x in dts)} s)"}
        line["rel_err_vs_fp64_sample"] = mode_errors(p, words, ref, [args.precision])[args.precision]
    if rank == 0 and world == 1 and not args.no_modes:
        # the other precisions on the same workload, each with its error
        # against the FP64 oracle on the sampled slice
        modes = {}
        errs = mode_errors(p, words, ref, [m for m in MODES if m != args.precision]) if ref is not None else {}
        for mode in MODES:
            if mode == args.precision:
                continue
            frac = C64_SLICE_FRACTION[args.workload] if mode == "c64" else 1
            modes[mode] = time_mode(p, dwords, out, stream, mode, slices, frac, nout)
            if mode in errs:
                modes[mode]["rel_err_vs_fp64_sample"] = errs[mode]
        line["precision_modes"] = modes
        if args.workload == "8x8" and not PLAN_CAP_AWARE:
            line["plan_variants"] = {"width_cap_aware_rewrites": cap_aware_variant(T, args, words, open_q, dwords,
                                                                                     out, stream, nout)}
            if PLAN_SEED == 1:
                # another search seed finds 9 fewer sliced indices at a lower
                # cost per slice under the same cap
                line["plan_variants"]["planner_seed_2"] = cap_aware_variant(T, args, words, open_q, dwords, out,
                                                                            stream, nout, cap_aware=0, seed=2)
        if args.workload == "8x8" and not args.no_6x6:
            line["workload_6x6"] = six_by_six_summary(T)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    # the workload's plan holds its arenas (most of the free HBM): release it
    # before the serving run sizes its budget
    del p
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_micro:
        line["pair_micro"] = pair_micro_summary(args)
    if rank == 0 and world == 1 and not args.no_serve:
        line["serving"] = serve_summary(args)
    if rank == 0:
        print(json.dumps(line))


def cap_aware_variant(T, args, words, open_q, dwords, out, stream, nout, cap_aware=1, seed=None):
    """The same workload planned another way -- with width-cap-aware subtree
    rewrites (fewer sliced indices under the 2^26 cap, more work per slice),
    or with another planner seed: one timed step of the bench precision, its
    error against the FP64 oracle on slice 0."""
    global PLAN_CAP_AWARE, PLAN_SEED
    keep, keep_seed = PLAN_CAP_AWARE, PLAN_SEED
    PLAN_CAP_AWARE = cap_aware
    if seed is not None:
        PLAN_SEED = seed
    try:
        _, _, p, _, _, _ = make_workload(T, 0)
    finally:
        PLAN_CAP_AWARE, PLAN_SEED = keep, keep_seed
    info = p.info()
    slices = min(SLICE_LIMIT, info["num_slices"])
    e = time_mode(p, dwords, out, stream, args.precision, slices, 1, nout)
    e.update({"plan_hash": hex(info["hash"]), "num_sliced": info["num_sliced"],
              "fidelity_fraction_log2": round(float(np.log2(slices)) - info["num_sliced"], 3),
              "cmac_per_slice_log2": round(float(np.log2(info["cmac_per_slice"])), 3),
              "max_log2_intermediate": info["max_log2_intermediate"]})
    if not args.no_cpu:
        ref, _, _ = oracle_reference(p, words, open_q)
        e["rel_err_vs_fp64_sample"] = mode_errors(p, words, ref, [args.precision])[args.precision]
    del p
    return e


def six_by_six_summary(T):
    """Every precision on the 6x6 configuration (1024 slices x 4 batches of 64
    amplitudes): one timed call each, error against the FP64 oracle on slice
    0 of batch 0."""
    import torch
    keep = {name: globals()[name] for name in ("ROWS", "COLS", "DEPTH", "CSEED", "NSLICED", "WIDTH_CAP", "NOPEN",
                                                "NBATCH", "BSEED", "PLAN_TRIALS", "SLICE_LIMIT", "WORKLOAD")}
    use_workload("6x6")
    try:
        c, net, p, words, open_q, plan_s = make_workload(T, 0)
        info = p.info()
        nout = NBATCH << info["num_open"]
        slices = info["num_slices"]
        stream = torch.cuda.Stream()
        dwords = torch.from_numpy(words.astype(np.int64)).cuda()
        out = torch.empty(nout * 2, dtype=torch.float64, device="cuda")
        ref, _, _ = oracle_reference(p, words, open_q)
        errs = mode_errors(p, words, ref, MODES)
        res = {"workload": WORKLOAD, "plan_hash": hex(info["hash"]),
               "cmac_per_slice_log2": round(float(np.log2(info["cmac_per_slice"])), 3), "modes": {}}
        for mode in MODES:
            frac = C64_SLICE_FRACTION["6x6"] if mode == "c64" else 1
            e = time_mode(p, dwords, out, stream, mode, slices, frac, nout)
            e["rel_err_vs_fp64_sample"] = errs[mode]
            res["modes"][mode] = e
        del p
        return res
    finally:
        globals().update(keep)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import paper_2110_14502_gb300 as T  # host planner only: supplies the schedule the oracle follows
    c, net, p, words, open_q, plan_s = make_workload(T, 0)
    info = p.info()
    for _ in range(args.warmup):
        cpu_oracle_sample(p, words, open_q, 0)
    tot, fl, times = 0.0, 0.0, []
    for s in range(args.steps):
        _, dt, cmac = cpu_oracle_sample(p, words, open_q, slice_id=s)
        tot += dt
        fl += 8 * cmac
        times.append(dt * 1e3)
    value = fl / tot / 1e12
    # one slice of a 2^k-amplitude batch is 1/slices of the work of those amplitudes
    slices = info["num_slices"] if SLICE_LIMIT < 0 else min(SLICE_LIMIT, info["num_slices"])
    amps_s = float(1 << info["num_open"]) / slices * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot * 1e3 / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded random circuit and bitstrings)",
            "config": {"workload": WORKLOAD, "precision": "fp64 oracle", "sample_per_step": "one slice of one batch"},
            "amplitudes_per_s": amps_s,
            "p50_ms": round(float(np.percentile(times, 50)), 1), "p99_ms": round(float(np.percentile(times, 99)), 1),
            "cpu_baseline": {"value": round(value, 6), "unit": "TFLOP/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                             "sample": f"per step: one slice of one {1 << info['num_open']}-amplitude batch, "
                                       "FP64 NumPy"},
            "e2e": {"value": round(value, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def micro_rows(shapes, precision, steps, warmup, random_layout, verbose=True):
    """Pairwise contraction microbenchmark rows: the fused tensor-core kernel
    (`precision`, its operand split included), the fused FP32 kernel and
    permute + cuBLAS cgemm on the same complex64 operands."""
    import torch
    import paper_2110_14502_gb300 as T
    import tn_inputs as I
    res = []
    for nm, nn, nk in shapes:
        rng = np.random.default_rng(3)
        labels = list(range(nm + nn + nk))
        M, N, K = labels[:nm], labels[nm:nm + nn], labels[nm + nn:]
        # planner-style layouts: contracted indices innermost, in one shared order
        perm_k = [int(x) for x in rng.permutation(K)]
        la = [int(x) for x in rng.permutation(M)] + perm_k
        lb = [int(x) for x in rng.permutation(N)] + perm_k
        lc = [int(x) for x in rng.permutation(M + N)]
        if random_layout:
            la = [int(x) for x in rng.permutation(M + K)]
            lb = [int(x) for x in rng.permutation(K + N)]
        A = torch.from_numpy(I.random_tensor(len(la), 31, np.complex64)).cuda()
        B = torch.from_numpy(I.random_tensor(len(lb), 32, np.complex64)).cuda()
        Cc = torch.empty(1 << len(lc), dtype=torch.complex64, device="cuda")
        flops = 8.0 * 2.0 ** (nm + nn + nk)
        tcp = precision if precision != "c64" else "split_bf16"
        row = {"shape": [nm, nn, nk], "tc_precision": tcp}
        algos = ["vector"] if (nn <= 4 and nk <= 4) else ["fused_tc", "gather_tc", "fused_simt", "unfused"]
        for algo in algos:
            prec = "c64"
            if algo == "fused_tc":
                prec = tcp
            elif algo == "gather_tc":
                prec = "split_bf16"
            for _ in range(warmup):
                T.contract_pair(A, la, B, lb, Cc, lc, precision=prec, algo=algo)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                T.contract_pair(A, la, B, lb, Cc, lc, precision=prec, algo=algo)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            row[algo] = {"ms": round(ms, 4), "tflops": round(flops / ms / 1e9, 2),
                         "gbs": round(8.0 * (2 ** len(la) + 2 ** len(lb) + 2 ** len(lc)) / ms / 1e6, 1)}
        res.append(row)
        if verbose:
            print(json.dumps(row), flush=True)
        del A, B, Cc
        torch.cuda.empty_cache()
    return res


def run_micro(args):
    """Pairwise contraction microbenchmark: fused kernels vs permute + cuBLAS."""
    shapes = [tuple(int(x) for x in args.shape.split(","))] if args.shape else \
        [(14, 12, 10), (12, 12, 12), (13, 13, 13), (19, 11, 11), (17, 13, 9), (26, 2, 2)]
    return micro_rows(shapes, args.precision, args.steps, args.warmup, args.random_layout)


# Pairwise microbenchmark of the bench line: complex64 operands of rank 20-30
# (2^20-2^30 elements), 4-14 contracted indices, random index orders on both
# operands and the output (log2 M, N, K).
PAIR_SHAPES = [(12, 12, 10), (14, 14, 12), (16, 6, 14), (15, 15, 5)]


def pair_micro_summary(args):
    rows = micro_rows(PAIR_SHAPES, args.precision, 2, 1, True, verbose=False)
    return {"operands": "complex64, rank 20-30, random index orders on both operands and the output, "
                        "N(0,1) entries; per tn_contract_pair call (the tensor-core arm includes its operand split)",
            "fused_tc": "tensor-core kernel in the bench precision", "fused_simt": "fused FP32 kernel (complex64)",
            "gather_tc": "tensor-core kernel gathering operands in its main loop (split bf16)",
            "unfused": "permute both operands, cuBLAS cgemm, permute the output (complex64)",
            "rows": rows}


def serve_workload(nreq, seed=5):
    """Request stream of the serving benchmark: grids R x C with R, C in [4, 7]
    and |R - C| <= 1, depth uniform in [10, 24], circuit seed 5 * 2^32 + id,
    m amplitudes log-uniform in [1, 4096] served as one bitstring with
    k = ceil(log2 m) open qubits; Poisson arrival gaps (unit rate)."""
    import tn_inputs as I
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(nreq):
        r = int(rng.integers(4, 8))
        c = int(np.clip(r + rng.integers(-1, 2), 4, 7))
        depth = int(rng.integers(10, 25))
        m = int(np.exp(rng.uniform(0, np.log(4096))))
        k = min(12, int(np.ceil(np.log2(max(m, 1)))))
        s = 5 * 2 ** 32 + i
        reqs.append(dict(rows=r, cols=c, depth=depth, seed=s, num_open=k,
                         bitstrings=I.bitstrings(r * c, 1, s)))
    gaps = rng.exponential(1.0, nreq)
    return reqs, gaps


def run_stream(T, srv, reqs, gaps=None, rate=None, keep=()):
    """Submits the requests (all at once, or at the Poisson arrival times
    gaps / rate) and waits for all of them: throughput, p50/p99 latency,
    refused count, and the amplitudes of the requests whose index is in
    `keep`."""
    t0 = time.time()
    tickets = []
    for i, r in enumerate(reqs):
        if rate:
            target = t0 + float(np.sum(gaps[:i + 1])) / rate
            while time.time() < target:
                time.sleep(0.0002)
        tickets.append(srv.submit(**r))
    lat, amps, refused, flops, kept, fractions, failed = [], 0, 0, 0.0, {}, [], []
    for i, t in enumerate(tickets):
        try:
            o, st = srv.wait(t)
            lat.append(st["submit_to_done_ms"])
            amps += o.size
            flops += st["flops"]
            if st["slice_fraction"] < 1.0:
                fractions.append(st["slice_fraction"])
            if i in keep:
                kept[i] = o
        except T.TnError as e:
            if e.status in (3, 6):  # TN_EHBM, TN_ETOOBIG: counted, never dropped silently
                refused += 1
            else:
                failed.append(str(e))
    dt = time.time() - t0
    res = {"seconds": round(dt, 3), "served": len(lat), "refused": refused,
           "amplitudes_per_s": round(amps / dt, 1), "tflops": round(flops / dt / 1e12, 3),
           "p50_ms": round(float(np.percentile(lat, 50)), 2) if lat else None,
           "p99_ms": round(float(np.percentile(lat, 99)), 2) if lat else None}
    if failed:  # any other error is reported, with its first message
        res["failed"] = len(failed)
        res["first_error"] = failed[0]
    if fractions:
        lf = np.log2(fractions)
        res["partial_fidelity"] = {"requests": len(fractions), "log2_fraction_min": round(float(lf.min()), 2),
                                   "log2_fraction_median": round(float(np.median(lf)), 2)}
    return res, kept


def serve_summary(args):
    """The serving stream (Poisson arrivals over random circuits, 4x4..7x7
    grids, depths 10-24, 1-4096 amplitudes each) on the plain path (one
    request at a time, one slice per launch group, complex64) and on the
    batched server (8 requests in flight, 64-slice quanta interleaved) in
    complex64, split bf16 and scaled fp16.  Each runs saturated (every request
    submitted at once: capacity) and with Poisson arrivals at 0.7 x the plain
    path's capacity (latency).  Served amplitudes of the 16-qubit requests are
    checked against the FP64 state vector."""
    import paper_2110_14502_gb300 as T
    import tn_inputs as I
    from oracle import circuit as OC
    from oracle import statevector as SV
    reqs, gaps = serve_workload(args.requests)
    common = dict(plan_trials=8, max_log2_cmac=args.cost_cap, max_log2_intermediate=27, planner_threads=16)
    small = [i for i, r in enumerate(reqs) if r["rows"] * r["cols"] <= 16][:8]
    refs = {}
    for i in small:
        r = reqs[i]
        n = r["rows"] * r["cols"]
        psi = SV.simulate(OC.random_circuit(r["rows"], r["cols"], r["depth"], r["seed"]), n)
        refs[i] = SV.amplitudes(psi, n, [I.bits_of(w, n) for w in r["bitstrings"]],
                                list(range(n - r["num_open"], n)))
    out = {"requests": args.requests, "cost_cap_log2_cmac": args.cost_cap,
           "stream": "seed 5; grids R x C, R, C in [4, 7], |R - C| <= 1; depth U[10, 24]; circuit seed 5 * 2^32 + id; "
                     "1-4096 amplitudes (log-uniform) as open-qubit batches",
           "error_check": f"{len(small)} served 16-qubit requests against the FP64 state vector"}
    # the plan cache is process-wide: the first pass plans every circuit
    warm = T.Server(max_inflight=8, slices_per_quantum=64, precision="c64", **common)
    out["first_pass_with_planning"], _ = run_stream(T, warm, reqs)
    warm.close()
    runs = (("plain_c64", dict(max_inflight=1, slices_per_quantum=1, precision="c64")),
            ("batched_c64", dict(max_inflight=8, slices_per_quantum=64, precision="c64")),
            ("batched_split_bf16", dict(max_inflight=8, slices_per_quantum=64, precision="split_bf16")),
            ("batched_scaled_fp16", dict(max_inflight=8, slices_per_quantum=64, precision="scaled_fp16")))
    rate = None
    for name, kw in runs:
        srv = T.Server(**kw, **common)
        try:
            sat, kept = run_stream(T, srv, reqs, keep=set(small))
            if rate is None:  # the plain path's capacity sets the arrival rate
                rate = 0.7 * (sat["served"] + sat["refused"]) / sat["seconds"]
                out["poisson_rate_req_per_s"] = round(rate, 2)
            poi, _ = run_stream(T, srv, reqs, gaps, rate)
        finally:
            srv.close()
        errs = [rel_err(kept[i].reshape(-1), refs[i].reshape(-1)) for i in small if i in kept]
        out[name] = {"saturated": sat, "poisson": poi,
                     "max_rel_err_vs_fp64": max(errs) if errs else None}
    # the same stream with over-cap requests served at partial fidelity (the
    # largest leading slice range that fits the cap) instead of refused
    srv = T.Server(max_inflight=8, slices_per_quantum=64, precision="split_bf16", over_cap_policy=1, **common)
    try:
        out["batched_split_bf16_over_cap_partial"], _ = run_stream(T, srv, reqs)
    finally:
        srv.close()
    return out


def run_serve(args):
    """Serving benchmark alone: the serving summary of the main line, with
    --requests requests."""
    import torch
    torch.cuda.set_device(0)
    s = serve_summary(args)
    line = {"metric": "serving amplitudes/s and p50/p99 latency",
            "value": s["batched_scaled_fp16"]["saturated"]["amplitudes_per_s"], "unit": "amplitudes/s", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "serving": s}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="split_fp16", choices=list(MODES))
    ap.add_argument("--micro", action="store_true")
    ap.add_argument("--shape", default=None)
    ap.add_argument("--random-layout", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--serve", action="store_true")
    ap.add_argument("--requests", type=int, default=300)
    ap.add_argument("--cost-cap", type=float, default=40.0)
    ap.add_argument("--workload", default="8x8", choices=list(WORKLOADS))
    ap.add_argument("--slices", type=int, default=0,
                    help="sum only the first N slices of the workload (profiling captures; 0: the workload's count)")
    ap.add_argument("--no-modes", action="store_true")
    ap.add_argument("--no-6x6", action="store_true")
    ap.add_argument("--no-micro", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="tune the tensor-core tiles per step in the first (warm-up) call")
    ap.add_argument("--plan-trials", type=int, default=0, help="order-search restarts (0: the workload's default)")
    ap.add_argument("--plan-seed", type=int, default=0, help="planner seed (0: the workload's default)")
    ap.add_argument("--plan-seeds", type=int, default=1,
                    help="search this many planner seeds from --plan-seed and keep the cheapest plan per slice")
    ap.add_argument("--bitstrings-hint", type=int, default=-1,
                    help="planner weight of bitstring-dependent steps (-1: the workload's default)")
    ap.add_argument("--cap-aware-rewrites", action="store_true",
                    help="plan with width-cap-aware subtree rewrites (fewer sliced indices under a width cap)")
    args = ap.parse_args()
    use_workload(args.workload)
    global PLAN_TRIALS, PLAN_SEED
    if args.plan_trials > 0:
        PLAN_TRIALS = args.plan_trials
    if args.plan_seed > 0:
        PLAN_SEED = args.plan_seed
    global PLAN_SEEDS
    PLAN_SEEDS = max(1, args.plan_seeds)
    global PLAN_HINT, PLAN_CAP_AWARE
    if args.bitstrings_hint >= 0:
        PLAN_HINT = args.bitstrings_hint
    if args.cap_aware_rewrites:
        PLAN_CAP_AWARE = 1
    if args.impl == "reference":
        run_reference(args)
    elif args.micro:
        run_micro(args)
    elif args.serve:
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
