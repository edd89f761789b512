"""Host-side logic of the library (no GPU): circuit protocol against the
oracle's independent generator, network and plan structure, plan determinism,
replay of plan trees by the oracle contractor, and argument validation."""
import ctypes as C
import re

import numpy as np
import pytest

import tn_inputs as I
from oracle import circuit as OC
from oracle import statevector as SV
from oracle import tn as OTN

from _lib import tnlib

KIND = {0: "sqrtx", 1: "sqrty", 2: "sqrtw", 3: "fsim"}


@pytest.mark.parametrize("rows,cols,depth,seed", [(4, 4, 8, 1), (6, 6, 16, 2), (3, 5, 7, 99), (8, 8, 20, 4)])
def test_library_circuit_equals_oracle_circuit(rows, cols, depth, seed):
    T = tnlib()
    lib_gates = T.random_circuit(rows, cols, depth, seed).gates()
    ora_gates = OC.random_circuit(rows, cols, depth, seed)
    assert len(lib_gates) == len(ora_gates)
    for (kind, q0, q1, th, ph, m), g in zip(lib_gates, ora_gates):
        assert KIND[kind] == g.kind
        assert (q0,) + ((q1,) if q1 >= 0 else ()) == tuple(g.qubits)
        assert np.allclose(m, g.matrix, atol=1e-15, rtol=0)


def test_network_counts():
    T = tnlib()
    c = T.random_circuit(3, 3, 4, 5)
    net = T.build_network(c, [7, 8])
    info = net.info()
    assert info["num_qubits"] == 9 and info["num_open"] == 2 and info["num_closed"] == 7
    # every wire segment is named (q, t) with t counting that qubit's gates
    wires = net.label_wires()
    per_q = {}
    for q, t in wires:
        per_q.setdefault(q, set()).add(t)
    gates = c.gates()
    for q in range(9):
        n_on_q = sum(1 for g in gates if q in (g[1], g[2]))
        assert per_q[q] == set(range(n_on_q + 1))


def _plan(T, rows, cols, depth, cseed, open_q=(), **kw):
    c = T.random_circuit(rows, cols, depth, cseed)
    net = T.build_network(c, list(open_q))
    return c, net, T.plan(net, **kw)


def test_plan_is_deterministic():
    T = tnlib()
    _, _, p1 = _plan(T, 4, 4, 8, 1, search_trials=16, seed=7, num_sliced=3)
    _, _, p2 = _plan(T, 4, 4, 8, 1, search_trials=16, seed=7, num_sliced=3)
    assert p1.serialize() == p2.serialize()
    assert p1.info()["hash"] == p2.info()["hash"]
    assert p1.info()["num_sliced"] == 3 and p1.info()["num_slices"] == 8


def test_plan_width_cap_and_errors():
    T = tnlib()
    _, _, p = _plan(T, 4, 5, 10, 3, open_q=(18, 19), max_log2_intermediate=8, search_trials=16)
    assert p.info()["max_log2_intermediate"] <= 8
    c = T.random_circuit(2, 2, 2, 1)
    net = T.build_network(c, [])
    with pytest.raises(T.TnError) as e:
        T.plan(net, num_sliced=1000)
    assert e.value.status == 1
    with pytest.raises(T.TnError):
        T.build_network(c, [0, 0])
    with pytest.raises(T.TnError):
        T.build_network(c, [5])


def _oracle_replay(T, rows, cols, depth, cseed, open_q, bits, **kw):
    """Contract the oracle's own network in the library plan's tree order."""
    from _replay import replay
    c, net, p = _plan(T, rows, cols, depth, cseed, open_q, **kw)
    gates = OC.random_circuit(rows, cols, depth, cseed)
    return replay(p, gates, rows * cols, bits, open_q), gates, p


@pytest.mark.parametrize("rows,cols,depth,seed,open_q", [(3, 3, 6, 1, ()), (3, 4, 8, 2, (10, 11)), (4, 4, 8, 3, (0, 15, 7))])
def test_oracle_replay_of_plan_tree_matches_statevector(rows, cols, depth, seed, open_q):
    T = tnlib()
    n = rows * cols
    bits = I.bits_of(I.bitstrings(n, 1, seed)[0], n)
    v, gates, _ = _oracle_replay(T, rows, cols, depth, seed, open_q, bits, search_trials=16, seed=1)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [bits], open_q)[0]
    assert np.linalg.norm(v - ref) <= 1e-12 * np.linalg.norm(ref)


def test_sliced_wires_name_internal_segments():
    T = tnlib()
    c, net, p = _plan(T, 4, 4, 8, 1, num_sliced=4, search_trials=16)
    sw = p.sliced_wires()
    assert len(sw) == 4 and len(set(sw)) == 4
    gates = c.gates()
    for q, t in sw:
        n_on_q = sum(1 for g in gates if q in (g[1], g[2]))
        assert 0 < t < n_on_q     # neither the input nor the output wire


def test_contract_rejects_bad_arguments_before_device_work():
    T = tnlib()
    _, _, p = _plan(T, 2, 2, 2, 1, search_trials=4)
    b = I.bitstrings(4, 2, 1)
    with pytest.raises(T.TnError) as e:
        p.contract_amplitudes(b, precision=99)
    assert e.value.status == 1
    with pytest.raises(T.TnError) as e:
        p.contract_amplitudes(b, slice_begin=5)
    assert e.value.status == 1


def test_library_exports_every_declared_symbol():
    T = tnlib()
    from paper_2110_14502_gb300 import _abi
    import os
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tn.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\*?\s+\*?(tn_[a-z0-9_]+)\s*\(", hdr, flags=re.M))
    assert len(names) >= 19
    h = C.CDLL(_abi.LIB_PATH)
    for nm in sorted(names):
        assert hasattr(h, nm), nm
    assert names <= set(_abi.SIGNATURES), names - set(_abi.SIGNATURES)


@pytest.mark.parametrize("rows,cols,depth,seed,open_q", [(3, 4, 8, 2, (10, 11)), (4, 4, 8, 1, ())])
def test_lattice_order_generator(rows, cols, depth, seed, open_q):
    """The PEPS-style lattice sweep (order_generator=1) gives a valid tree --
    its oracle replay equals the state vector -- and on these random fSim
    circuits costs at least as many complex MACs as the default search."""
    T = tnlib()
    n = rows * cols
    bits = I.bits_of(I.bitstrings(n, 1, seed)[0], n)
    v, gates, p = _oracle_replay(T, rows, cols, depth, seed, open_q, bits, search_trials=4, seed=1,
                                 order_generator=1)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [bits], open_q)[0]
    assert np.linalg.norm(v - ref) <= 1e-12 * np.linalg.norm(ref)
    _, _, p0 = _plan(T, rows, cols, depth, seed, open_q, search_trials=64, seed=1)
    assert p.info()["log2_cmac_total"] >= p0.info()["log2_cmac_total"] - 1e-9
    _, _, p2 = _plan(T, rows, cols, depth, seed, open_q, search_trials=4, seed=1, order_generator=1)
    assert p2.info()["hash"] == p.info()["hash"]


def test_planner_options_default_to_the_plain_search():
    """bitstrings_hint 0 and 1 and order_generator 0 are the plain search:
    the same plan bytes as the defaults; a hint above 1 may change the plan
    but keeps it valid."""
    T = tnlib()
    c = T.random_circuit(5, 5, 12, 3)
    net = T.build_network(c, [20, 21, 22])
    base = T.plan(net, num_sliced=4, search_trials=16, seed=2)
    for kw in (dict(bitstrings_hint=0), dict(bitstrings_hint=1), dict(order_generator=0)):
        p = T.plan(net, num_sliced=4, search_trials=16, seed=2, **kw)
        assert p.serialize() == base.serialize(), kw
    p4 = T.plan(net, num_sliced=4, search_trials=16, seed=2, bitstrings_hint=4)
    assert p4.info()["num_sliced"] == 4 and p4.info()["num_qubits"] == 25


@pytest.mark.parametrize("workload,hash_,log2_cmac,sliced,width,nb,first_open", [
    ("8x8", "0x5973de292b52ff33", 35.846, 80, 24, 1, 54),
    ("6x6", "0x3e0860a7cb099543", 36.525, 10, 26, 4, 30)])
def test_bench_workload_plan_is_reproducible(workload, hash_, log2_cmac, sliced, width, nb, first_open):
    """The planner is deterministic host code: the bench's workloads plan to
    the same tree, hash and work on any host (the hashes and the work below
    are the ones the bench reports on the GPU machine's Arm host)."""
    import bench
    T = tnlib()
    bench.use_workload(workload)
    try:
        _, _, p, words, open_q, _ = bench.make_workload(T, 0)
    finally:
        bench.use_workload("8x8")
    info = p.info()
    assert hex(info["hash"]) == hash_
    assert round(float(np.log2(info["cmac_per_slice"])), 3) == log2_cmac
    assert info["num_sliced"] == sliced and info["max_log2_intermediate"] == width
    assert words.shape[0] == nb and open_q == list(range(first_open, first_open + len(open_q)))


def test_size_limits_fail_before_any_work():
    """Sizes whose products would overflow 64-bit offsets are rejected with
    TN_EINVAL on the host: a grid side far above 64, more than 2^40 amplitudes
    in one call, a tree buffer shorter than the plan's steps."""
    T = tnlib()
    from paper_2110_14502_gb300 import _abi
    L = _abi.lib()
    h = C.c_void_p()
    assert L.tn_random_circuit(1 << 20, 1 << 20, 4, 1, C.byref(h)) == 1
    assert "bad grid" in L.tn_last_error().decode()
    _, _, p = _plan(T, 2, 3, 4, 1, open_q=(4, 5), search_trials=4)
    words = np.zeros(1, dtype=np.uint64)
    out = np.zeros(2, dtype=np.float64)
    st = L.tn_contract_amplitudes(p._h, words.ctypes.data_as(C.c_void_p), 1 << 39, out.ctypes.data_as(C.c_void_p),
                                  None, None)
    assert st == 1 and "2^40" in L.tn_last_error().decode()
    nl = p.info()["num_leaves"]
    raw = np.zeros(4096, dtype=np.int32)
    tree = np.zeros(2 * (nl - 1) - 1, dtype=np.int32)
    st = L.tn_plan_tree(p._h, raw.ctypes.data_as(C.POINTER(C.c_int32)), raw.size,
                        tree.ctypes.data_as(C.POINTER(C.c_int32)), tree.size)
    assert st == 1 and "capacity too small" in L.tn_last_error().decode()
    assert _abi.STATUS[10] == "TN_EINTERNAL"


def test_header_is_plain_c_and_the_library_links_from_c(tmp_path):
    """include/tn.h compiles as strict C99, and a C program linked against the
    library plans the same bytes (hash) as the Python binding."""
    import os
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    T = tnlib()
    from paper_2110_14502_gb300 import _abi
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(_abi.LIB_PATH)
    exe = str(tmp_path / "c_abi_host")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(root, "include"),
           os.path.join(root, "tests", "c_abi_host.c"), "-o", exe, "-L", libdir, "-ltn", f"-Wl,-rpath,{libdir}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    fields = dict(kv.split("=") for kv in r.stdout.split())
    c = T.random_circuit(4, 4, 8, 1)
    p = T.plan(T.build_network(c, [14, 15]), num_sliced=2, search_trials=8, seed=3)
    assert int(fields["hash"], 16) == p.info()["hash"]
    assert int(fields["slices"]) == 4 and int(fields["bytes"]) == len(p.serialize())


def test_cost_cap_premise_of_the_partial_fidelity_serving_test():
    """Host facts the partial-fidelity serving test relies on: the 4x5
    depth-12 circuit (seed 21, 3 open, width 2^12, 8 trials, seed 1) plans to
    2^26.38 CMAC in 2^8 slices; a 2^25.3 cap refuses it, and so does the cap a
    fidelity-0.75 request gets (25.3 + log2(4/3)); the fidelity-0.25 cap
    (27.3) plans it."""
    import math
    T = tnlib()
    net = T.build_network(T.random_circuit(4, 5, 12, 21), [17, 18, 19])
    kw = dict(max_log2_intermediate=12, search_trials=8, seed=1)
    for cap in (25.3, 25.3 + math.log2(4 / 3)):
        with pytest.raises(T.TnError) as e:
            T.plan(net, max_log2_cmac=cap, **kw)
        assert e.value.status == 6
    info = T.plan(net, max_log2_cmac=27.3, **kw).info()
    assert info["num_sliced"] == 8 and abs(info["log2_cmac_total"] - 26.382) < 1e-3
    assert math.log2(64 * info["cmac_per_slice"]) <= 25.3


@pytest.mark.parametrize("rows,cols,depth,seed,open_q,ns", [(3, 4, 8, 2, (10, 11), 3), (4, 4, 8, 3, (), 4)])
def test_sliced_plan_replayed_slice_by_slice_sums_to_the_statevector(rows, cols, depth, seed, open_q, ns):
    """Slicing is exact: fixing the plan's sliced wires to the bits of each
    slice id (bit j of s for sliced index j) and contracting every slice in
    the plan's order with the oracle, the FP64 sum over the 2^S slices is the
    state-vector amplitude; no single slice is."""
    T = tnlib()
    from _replay import replay
    n = rows * cols
    c, net, p = _plan(T, rows, cols, depth, seed, open_q, num_sliced=ns, search_trials=16, seed=1)
    gates = OC.random_circuit(rows, cols, depth, seed)
    bits = I.bits_of(I.bitstrings(n, 1, seed)[0], n)
    wires = p.sliced_wires()
    assert len(wires) == ns
    parts = [replay(p, gates, n, bits, open_q, {wires[j]: (s >> j) & 1 for j in range(ns)}) for s in range(1 << ns)]
    ref = SV.amplitudes(SV.simulate(gates, n), n, [bits], open_q)[0]
    total = np.sum(parts, axis=0)
    assert np.linalg.norm(total - ref) <= 1e-12 * np.linalg.norm(ref)
    assert all(np.linalg.norm(x - ref) > 1e-6 * np.linalg.norm(ref) for x in parts)


def test_binding_checks_buffers_before_passing_pointers():
    """The C ABI cannot see buffer sizes, so the binding checks side, dtype,
    contiguity and size of every buffer it passes as a raw pointer."""
    import torch
    T = tnlib()
    from paper_2110_14502_gb300._abi import require_buffer
    _, _, p = _plan(T, 2, 3, 4, 1, open_q=(4, 5), search_trials=4)
    with pytest.raises(T.TnError) as e:
        p.contract_amplitudes(np.zeros((2, 2), dtype=np.uint64))      # two words per bitstring for 6 qubits
    assert e.value.status == 1
    words = np.zeros((3, 1), dtype=np.uint64)
    for out in (np.zeros((3, 4), np.complex64), np.zeros((2, 4), np.complex128), np.zeros((4, 3), np.complex128).T):
        with pytest.raises(T.TnError) as e:                          # host `out`: complex128, 3 x 2^2, contiguous
            p.contract_amplitudes(words, out=out)
        assert e.value.status == 1 and "out must be" in str(e.value)
    a = torch.zeros(4, dtype=torch.complex64)                          # host tensors: the pair path is device-only
    with pytest.raises(T.TnError) as e:
        T.contract_pair(a, [0, 1], a, [1, 2], a, [0, 2])
    assert e.value.status == 1 and "CUDA tensor" in str(e.value)
    require_buffer(np.zeros(4, np.complex64), "x", 32, False, ("complex64",))
    for bad in (np.zeros(3, np.complex64), np.zeros(4, np.complex128), np.zeros((4, 2), np.complex64)[:, 0]):
        with pytest.raises(T.TnError):
            require_buffer(bad, "x", 32, False, ("complex64",))
    with pytest.raises(T.TnError):
        require_buffer(np.zeros(4, np.complex64), "x", 32, True, ("complex64",))


@pytest.mark.parametrize("rows,cols,depth,seed,open_q,kw", [
    (3, 3, 5, 11, (8,), dict(num_sliced=2)),
    (4, 4, 8, 12, (), dict(max_log2_intermediate=9)),
    (3, 5, 9, 13, (12, 13, 14), dict(num_sliced=3, order_generator=1)),
    (5, 4, 10, 14, (18, 19), dict(max_log2_intermediate=11, bitstrings_hint=8)),
])
def test_plan_tree_is_a_binary_tree_over_the_leaves(rows, cols, depth, seed, open_q, kw):
    """Structure of any plan: L - 1 steps whose operands are SSA ids, each
    leaf and each intermediate consumed exactly once, every operand defined
    before its use, the last step the root; the leaves' raw gate lists
    partition the circuit's gates and input vectors; the width cap holds."""
    T = tnlib()
    n = rows * cols
    c, net, p = _plan(T, rows, cols, depth, seed, open_q, search_trials=8, seed=5, **kw)
    info = p.info()
    L = info["num_leaves"]
    ng = len(c.gates())
    leaves, pairs = p.tree(ng, n)
    assert len(leaves) == L and len(pairs) == L - 1 == info["num_steps"]
    used = []
    for i, (a, b) in enumerate(pairs):
        assert a != b and max(a, b) < L + i          # defined before use
        used += [a, b]
    assert sorted(used) == list(range(L + len(pairs) - 1))   # everything but the root, once
    raws = sorted(r for lf in leaves for r in lf)
    assert raws == list(range(ng + n))
    if kw.get("max_log2_intermediate"):
        assert info["max_log2_intermediate"] <= kw["max_log2_intermediate"]


def test_cap_aware_rewrites_keep_the_width_cap_and_cut_the_8x8_cost():
    """Subtree rewrites after slicing may widen an intermediate beyond the
    per-slice width cap; a trial whose rewrite did so loses to any trial that
    kept the cap.  Constraining the rewrites (cap_aware_rewrites=1) keeps
    every trial valid: on the 8x8 depth-(1+20+1) network under a 2^26 cap the
    plan needs 12 fewer sliced indices and 2^10 less total work.  The default
    search keeps its plans (the bench's 8x8 plan hash below) and falls back to
    constrained rewrites only when no trial met the cap."""
    T = tnlib()
    net = T.build_network(T.random_circuit(8, 8, 20, 4), list(range(54, 64)))
    kw = dict(max_log2_intermediate=26, search_trials=16, seed=1)
    plain = T.plan(net, **kw).info()
    aware = T.plan(net, cap_aware_rewrites=1, **kw).info()
    assert hex(plain["hash"]) == "0x5973de292b52ff33"
    assert plain["max_log2_intermediate"] <= 26 and aware["max_log2_intermediate"] <= 26
    assert aware["num_sliced"] <= plain["num_sliced"] - 12
    assert aware["log2_cmac_total"] <= plain["log2_cmac_total"] - 10
    with pytest.raises(T.TnError) as e:
        T.plan(net, cap_aware_rewrites=2, **kw)
    assert e.value.status == 1


def _check_layout(tensors, size, info):
    """Memory layout invariants of a plan (see test below); returns the
    number of tensors checked per memory."""
    L = info["num_leaves"]
    assert len(tensors) == L + info["num_steps"]
    # the tree: every tensor but the root consumed once, by a later step
    assert sum(t["consumer"] < 0 for t in tensors) == 1
    for x, t in enumerate(tensors):
        assert (t["producer"] < 0) == (x < L)
        assert t["consumer"] < 0 or t["consumer"] > max(t["producer"], -1)
    # execution order: phase 0 steps, then phase 1, then phase 2, each in step order
    order = sorted(range(info["num_steps"]), key=lambda s: (tensors[L + s]["phase"], s))
    when = {s: i for i, s in enumerate(order)}
    END = len(order)
    spaces = {"leaf_store": [], "invariant": [], "slice_arena": [], "pair_arena": []}
    for x, t in enumerate(tensors):
        n = 1 << t["log2_elems"]
        assert t["offset"] % 32 == 0
        if x < L:
            spaces["leaf_store"].append((t["store_offset"], 1 << t["store_log2"], -1, END))
            assert t["store_offset"] % 32 == 0 and t["store_log2"] >= t["log2_elems"]
            if t["phase"] == 0:
                assert t["offset"] == t["store_offset"]
                continue
        born = -1 if x < L else when[t["producer"]]
        c = t["consumer"]
        # a tensor is freed when a step of its own phase consumes it; one read by
        # a later phase (or the root) stays until the end
        dies = when[c] if c >= 0 and tensors[L + c]["phase"] == t["phase"] else END
        space = ("invariant", "slice_arena", "pair_arena")[t["phase"]]
        spaces[space].append((t["offset"], n, born, dies))
    for name, blocks in spaces.items():
        for off, n, _, _ in blocks:
            assert 0 <= off and off + n <= size[name], name
        for i in range(len(blocks)):
            for j in range(i + 1, len(blocks)):
                (o1, n1, b1, d1), (o2, n2, b2, d2) = blocks[i], blocks[j]
                live_together = not (d1 < b2 or d2 < b1)
                apart = o1 + n1 <= o2 or o2 + n2 <= o1
                assert apart or not live_together, (name, blocks[i], blocks[j])
    return {k: len(v) for k, v in spaces.items()}


@pytest.mark.parametrize("rows,cols,depth,seed,open_q,kw", [
    (3, 4, 8, 2, (10, 11), dict(num_sliced=3)),
    (4, 4, 10, 5, (15, 14), dict(num_sliced=4)),
    (4, 5, 12, 21, (17, 18, 19), dict(max_log2_intermediate=12)),
    (5, 5, 12, 3, (22, 23, 24), dict(max_log2_intermediate=14, bitstrings_hint=4)),
    (6, 6, 16, 2, tuple(range(30, 36)), dict(num_sliced=10, search_trials=64, seed=1)),
])
def test_plan_memory_layout_is_disjoint_while_live(rows, cols, depth, seed, open_q, kw):
    """The planner's HBM layout: leaves packed in the leaf store, phase-0
    results in the invariant store without reuse, slice-only and per-unit
    tensors in their arenas by first-fit over liveness.  Every tensor is
    32-element aligned and inside its memory, and no two tensors of one
    memory overlap while both are live (a step's output is live together with
    its inputs)."""
    T = tnlib()
    kw = dict(dict(search_trials=16, seed=3), **kw)
    _, _, p = _plan(T, rows, cols, depth, seed, open_q, **kw)
    counts = _check_layout(*p.layout(), p.info())
    assert counts["leaf_store"] == p.info()["num_leaves"]


def test_layout_check_catches_an_overlap():
    """The layout check is not vacuous: moving a step's output onto one of its
    own inputs, or past the end of its arena, fails it."""
    T = tnlib()
    _, _, p = _plan(T, 4, 4, 10, 5, (15, 14), num_sliced=4, search_trials=16, seed=3)
    tensors, size = p.layout()
    info = p.info()
    L = info["num_leaves"]
    _check_layout(tensors, size, info)
    s = next(s for s in range(info["num_steps"])
             if tensors[L + s]["phase"] == 2 and any(t["consumer"] == s and t["phase"] == 2 for t in tensors))
    src = next(t for t in tensors if t["consumer"] == s and t["phase"] == 2)
    bad = [dict(t) for t in tensors]
    bad[L + s]["offset"] = src["offset"]
    with pytest.raises(AssertionError):
        _check_layout(bad, size, info)
    bad = [dict(t) for t in tensors]
    bad[L + s]["offset"] = size["pair_arena"]
    with pytest.raises(AssertionError):
        _check_layout(bad, size, info)


def _random_configs(count, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        rows, cols = int(rng.integers(1, 4)), int(rng.integers(2, 5))
        n = rows * cols
        depth = int(rng.integers(0, 9))
        k = int(rng.integers(0, min(n, 4) + 1))
        open_q = tuple(sorted(int(q) for q in rng.choice(n, size=k, replace=False)))
        kw = dict(search_trials=int(rng.integers(1, 9)), seed=int(rng.integers(1, 1000)),
                  order_generator=int(rng.integers(0, 2)), bitstrings_hint=int(rng.integers(0, 5)))
        out.append((rows, cols, depth, int(rng.integers(1, 10 ** 6)), open_q, int(rng.integers(0, 4)), kw))
    return out


@pytest.mark.parametrize("rows,cols,depth,cseed,open_q,ns,kw", _random_configs(16))
def test_random_small_plans_are_exact(rows, cols, depth, cseed, open_q, ns, kw):
    """Sixteen seeded random small circuits (1..3 x 2..4 grids, depth 0..8,
    0..4 open qubits at random positions, up to 3 sliced indices (as many as
    the network has), random planner options): the plan's tree replayed by
    the oracle and summed over all 2^S slice assignments equals the state
    vector, and the memory layout holds."""
    T = tnlib()
    from _replay import replay
    n = rows * cols
    c = T.random_circuit(rows, cols, depth, cseed)
    net = T.build_network(c, list(open_q))
    while True:                                         # the most sliced indices <= ns the network has
        try:
            p = T.plan(net, num_sliced=ns, **kw)
            break
        except T.TnError as e:
            assert e.status == 1 and "exceeds" in str(e) and ns > 0, str(e)
            ns -= 1
    gates = OC.random_circuit(rows, cols, depth, cseed)
    bits = I.bits_of(I.bitstrings(n, 1, cseed)[0], n)
    wires = p.sliced_wires()
    S = len(wires)
    total = sum(replay(p, gates, n, bits, open_q, {wires[j]: (s >> j) & 1 for j in range(S)} if S else None)
                for s in range(1 << S))
    ref = SV.amplitudes(SV.simulate(gates, n), n, [bits], open_q)[0]
    assert np.linalg.norm(total - ref) <= 1e-12 * max(np.linalg.norm(ref), 1e-300)
    _check_layout(*p.layout(), p.info())


def test_step_shapes_account_for_the_counted_work():
    """The GEMM shape of every step in the layout: its output holds M N
    elements, its operands M K and K N (in either order), and the counted
    work of a slice, 2^(m+n+k) complex MACs summed over the steps, is the
    plan's cmac_per_slice exactly (the flops the bench reports are these).
    Vector-like steps are the narrow ones."""
    T = tnlib()
    import bench
    _, _, p, _, _, _ = bench.make_workload(T, 0)
    tensors, _ = p.layout()
    info = p.info()
    L = info["num_leaves"]
    total = 0.0
    for s, t in enumerate(tensors[L:]):
        m, n, k = t["log2_m"], t["log2_n"], t["log2_k"]
        assert t["log2_elems"] == m + n
        ops = sorted(tensors[x]["log2_elems"] for x in range(len(tensors)) if tensors[x]["consumer"] == s)
        assert ops == sorted([m + k, k + n]), s
        assert t["step_class"] in (0, 1)
        if t["step_class"] == 1:
            assert (n <= 4 and k <= 4) or (n <= 3 and k <= 7)
        total += 2.0 ** (m + n + k)
    assert total == info["cmac_per_slice"]
    assert info["num_vector_steps"] == sum(t["step_class"] == 1 for t in tensors[L:])


def test_plan_hash_is_fnv1a_of_the_serialized_bytes():
    """The plan hash is FNV-1a 64 (offset basis 0xcbf29ce484222325, prime
    0x100000001b3, Fowler-Noll-Vo) over the serialized plan, computed here
    independently; the bytes start with the format tag."""
    T = tnlib()
    _, _, p = _plan(T, 4, 4, 8, 1, open_q=(14, 15), num_sliced=2, search_trials=8, seed=3)
    b = p.serialize()
    h = 0xcbf29ce484222325
    for x in b:
        h = ((h ^ x) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    assert h == p.info()["hash"]
    assert b[:8] == b"TNPLAN01"


def test_step_precision_and_precision_analysis_arguments_are_checked():
    """A per-step precision outside TN_PREC_* and the pre-analysis' bad
    arguments fail with TN_EINVAL on the host, before any device work."""
    T = tnlib()
    from paper_2110_14502_gb300 import _abi
    L = _abi.lib()
    _, _, p = _plan(T, 3, 3, 6, 1, open_q=(7, 8), num_sliced=2, search_trials=4)
    ns = p.info()["num_steps"]
    words = np.zeros(1, dtype=np.uint64)
    out = np.zeros(8, dtype=np.complex128)
    bad = np.full(ns, 7, dtype=np.int8)
    o = _abi.ExecOpts()
    o.slice_count = -1
    o.step_precision = bad.ctypes.data
    st = L.tn_contract_amplitudes(p._h, words.ctypes.data_as(C.c_void_p), 1, out.ctypes.data_as(C.c_void_p),
                                  C.byref(o), None)
    assert st == 1 and "unknown precision 7" in L.tn_last_error().decode()
    sp = np.zeros(ns, dtype=np.int8)
    rep = _abi.PrecisionReport()
    for args, msg in (((words.ctypes.data, 1, 4, 0, 2, 1e-3), "16-bit"),       # c64 is not a 16-bit precision
                      ((words.ctypes.data, 1, 4, 4, 2, 0.0), "target"),
                      ((words.ctypes.data, 0, 4, 4, 2, 1e-3), "probe bitstrings"),
                      ((words.ctypes.data, 1, 5, 4, 2, 1e-3), "outside"),      # 2 sliced indices: 4 slices
                      ((None, 1, 4, 4, 2, 1e-3), "NULL")):
        st = L.tn_precision_analysis(p._h, *args, sp.ctypes.data, C.byref(rep))
        assert st == 1 and msg in L.tn_last_error().decode(), (args, L.tn_last_error())


@pytest.mark.parametrize("rows,cols,depth,seed,open_q,S", [(3, 3, 6, 1, (), 0), (3, 4, 8, 2, (10, 11), 3),
                                                           (4, 4, 8, 3, (0, 15, 7), 4)])
def test_split_diagonal_plan_replays_to_the_statevector(rows, cols, depth, seed, open_q, S):
    """TN_NET_SPLIT_DIAGONAL: the library's network with every fSim(pi/2, pi/6)
    turned into a wire swap plus a bond, planned and sliced; the oracle's own
    hyperedge network (oracle.hyper) contracted in the plan's tree order and
    summed over every assignment of the sliced indices (named by wire, bonds
    by gate) equals the state vector."""
    from _replay import replay
    T = tnlib()
    n = rows * cols
    c = T.random_circuit(rows, cols, depth, seed)
    net = T.build_network(c, list(open_q), split_diagonal=True)
    p = T.plan(net, num_sliced=S, search_trials=16, seed=1)
    assert p.info()["num_sliced"] == S
    gates = OC.random_circuit(rows, cols, depth, seed)
    bits = I.bits_of(I.bitstrings(n, 1, seed)[0], n)
    wires = p.sliced_wires()
    total = 0
    for s in range(1 << S):
        fixed = {w: (s >> j) & 1 for j, w in enumerate(wires)}
        total = total + replay(p, gates, n, bits, open_q, fixed, split=True)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [bits], open_q)[0]
    assert np.linalg.norm(total - ref) <= 1e-12 * np.linalg.norm(ref)


def test_split_diagonal_costs_against_the_plain_network():
    """The measured effect of the diagonal decomposition on the planner's cost
    (log2 complex MACs per slice, same search): about even on the 4x4, worse on
    the 6x6 with 10 sliced indices, because each swap carries a qubit's wire to
    its neighbour's site and the lattice's cuts grow."""
    T = tnlib()
    res = {}
    for split in (False, True):
        c = T.random_circuit(6, 6, 16, 2)
        p = T.plan(T.build_network(c, list(range(30, 36)), split_diagonal=split), num_sliced=10, search_trials=64,
                   seed=1)
        res[split] = round(float(np.log2(p.info()["cmac_per_slice"])), 2)
    assert res == {False: 36.53, True: 39.54}, res


def test_plans_with_more_than_62_sliced_indices_address_a_leading_slice_range():
    """With S >= 62 sliced indices the slice ids (int64) address the first
    2^62 slices (bit j of the id fixes sliced index j; higher indices stay 0):
    num_slices says so, a range inside it passes the host checks and one
    beyond it fails with TN_EINVAL before any device work."""
    T = tnlib()
    from paper_2110_14502_gb300 import _abi
    L = _abi.lib()
    p = T.plan(T.build_network(T.random_circuit(8, 8, 20, 4), list(range(54, 64))), max_log2_intermediate=26,
               search_trials=16, seed=1, cap_aware_rewrites=1)
    info = p.info()
    assert info["num_sliced"] == 68 and info["num_slices"] == 1 << 62
    assert abs(info["log2_cmac_total"] - (68 + np.log2(info["cmac_per_slice"]))) < 1e-9
    words = np.zeros((1, 1), dtype=np.uint64)
    out = np.zeros(2 << 10, dtype=np.float64)
    o = _abi.ExecOpts()
    o.slice_begin = (1 << 62) - 1
    o.slice_count = 2
    st = L.tn_contract_amplitudes(p._h, words.ctypes.data_as(C.c_void_p), 1, out.ctypes.data_as(C.c_void_p),
                                  C.byref(o), None)
    assert st == 1 and "outside [0, 4611686018427387904)" in L.tn_last_error().decode()


def test_planner_seed_2_plan_of_the_8x8_network():
    """The bench line's seed-2 plan variant: the same search (16 trials, 2^26
    cap) from seed 2 plans the 8x8 depth-(1+20+1) network with 9 fewer sliced
    indices and a lower cost per slice than the default seed, within the cap
    (the hash and work the bench reports on the GPU machine's Arm host)."""
    T = tnlib()
    net = T.build_network(T.random_circuit(8, 8, 20, 4), list(range(54, 64)))
    kw = dict(max_log2_intermediate=26, search_trials=16)
    one = T.plan(net, seed=1, **kw).info()
    two = T.plan(net, seed=2, **kw).info()
    assert hex(two["hash"]) == "0x5f3438fc5f089094"
    assert two["num_sliced"] == 71 and one["num_sliced"] == 80
    assert round(float(np.log2(two["cmac_per_slice"])), 3) == 35.76
    assert two["cmac_per_slice"] < one["cmac_per_slice"]
    assert two["log2_cmac_total"] <= one["log2_cmac_total"] - 9
    assert two["max_log2_intermediate"] <= 26


def test_bench_plan_search_over_seeds_keeps_the_cheapest_per_slice():
    """bench.py --plan-seeds: of the plans from several planner seeds the one
    with the least work per slice is kept (the benchmark sums a fixed number
    of slices).  On the 8x8 network, seeds 20-27 include seed 25's plan, the
    cheapest per slice of seeds 1-40 (74 sliced indices, 2^35.362 per slice;
    259.6 amplitudes/s on the GPU against 196 for the default seed-1 plan)."""
    import bench
    T = tnlib()
    bench.use_workload("8x8")
    c = T.random_circuit(bench.ROWS, bench.COLS, bench.DEPTH, bench.CSEED)
    n = bench.ROWS * bench.COLS
    net = T.build_network(c, list(range(n - bench.NOPEN, n)))
    best = bench.best_plan_of_seeds(T, net, range(20, 28)).info()
    assert hex(best["hash"]) == "0x85af835ff396f738"
    assert best["num_sliced"] == 74 and round(float(np.log2(best["cmac_per_slice"])), 3) == 35.362
    one = bench.best_plan_of_seeds(T, net, [1]).info()
    assert hex(one["hash"]) == "0x5973de292b52ff33"
