"""End-to-end amplitude parity of the CUDA path against the CPU oracle.

Bounds: relative L2 error of an amplitude batch <= 1e-5 for complex64
(the tolerance of the plain complex64 path)."""
import numpy as np
import pytest

import tn_inputs as I
from oracle import circuit as OC
from oracle import statevector as SV
from oracle import tn as OTN

from _lib import tnlib
from _replay import replay

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _setup(T, rows, cols, depth, cseed, open_q=(), **kw):
    c = T.random_circuit(rows, cols, depth, cseed)
    net = T.build_network(c, list(open_q))
    return T.plan(net, **kw)


def test_config_4x4_depth8_64_bitstrings_vs_statevector():
    """4x4 grid, depth 1+8+1, seed 1, 64 bitstrings, complex64 unsliced."""
    T = tnlib()
    n = 16
    p = _setup(T, 4, 4, 8, 1, search_trials=64, seed=1)
    words = I.bitstrings(n, 64, 1)
    got = p.contract_amplitudes(words)
    gates = OC.random_circuit(4, 4, 8, 1)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in words])
    assert got.shape == (64, 1)
    assert rel(got, ref) <= 1e-5


@pytest.mark.parametrize("rows,cols,depth,seed,open_q,S", [
    (3, 4, 10, 2, (10, 11, 3), 0),
    (4, 4, 10, 5, (15, 14), 4),
    (4, 5, 12, 6, (14, 15, 16, 17, 18, 19), 6),
    (2, 3, 4, 8, (), 2),
    (1, 1, 3, 9, (0,), 0),
    (1, 2, 0, 9, (), 0),
])
def test_open_and_sliced_vs_statevector(rows, cols, depth, seed, open_q, S):
    T = tnlib()
    n = rows * cols
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=S, search_trials=32, seed=3)
    assert p.info()["num_sliced"] == S
    words = I.bitstrings(n, 5, seed)
    got = p.contract_amplitudes(words)
    gates = OC.random_circuit(rows, cols, depth, seed)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in words], open_q)
    assert rel(got, ref) <= 1e-5


def test_slice_ids_map_to_the_oracle_assignment():
    """Slice s fixes sliced wire j to bit j of s: per-slice values and a
    ragged subset sum agree with the oracle's contraction of the same
    assignment."""
    T = tnlib()
    rows, cols, depth, seed, open_q = 4, 4, 10, 11, (12, 13)
    n = rows * cols
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=5, search_trials=32, seed=2)
    wires = p.sliced_wires()
    words = I.bitstrings(n, 2, seed)
    gates = OC.random_circuit(rows, cols, depth, seed)
    for bi, w in enumerate(words):
        bits = I.bits_of(w, n)
        net = OTN.circuit_network(gates, n, bits, open_q)
        for s in (0, 1, 6, 17, 31):
            got = p.contract_amplitudes(words[bi:bi + 1], slice_begin=s, slice_count=1)[0]
            ref = OTN.contract_slice(net, wires, s)
            assert rel(got, ref) <= 1e-5, (bi, s)
        got = p.contract_amplitudes(words[bi:bi + 1], slice_begin=3, slice_count=11)[0]
        ref = OTN.contract_sliced(net, wires, range(3, 14))
        assert rel(got, ref) <= 1e-5


def test_group_size_does_not_change_the_sum():
    """The FP64 cross-slice sum runs in unit order, so any grouping gives
    bit-identical results."""
    T = tnlib()
    p = _setup(T, 4, 4, 10, 5, (15, 14), num_sliced=4, search_trials=16, seed=3)
    words = I.bitstrings(16, 3, 5)
    r0 = p.contract_amplitudes(words, units_per_group=1)
    for g in (3, 7, 48, 0):
        assert np.array_equal(p.contract_amplitudes(words, units_per_group=g), r0)


def test_device_io_matches_host_io():
    import torch
    T = tnlib()
    p = _setup(T, 4, 4, 8, 3, (0, 1), num_sliced=2, search_trials=16, seed=3)
    words = I.bitstrings(16, 6, 3)
    host = p.contract_amplitudes(words)
    dw = torch.from_numpy(words.astype(np.int64)).cuda()
    out = torch.empty(6 * 4 * 2, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    p.contract_amplitudes(dw, out=out, stream=s)
    torch.cuda.synchronize()
    dev = out.cpu().numpy().view(np.complex128).reshape(6, 4)
    assert np.array_equal(dev, host)


def test_full_size_6x6_sampled_slices_vs_oracle():
    """6x6 grid (36 qubits), depth 1+16+1, seed 2, 10 sliced indices, six
    open qubits (the last six): two sampled slices of one bitstring batch
    against the oracle's FP64 contraction of the same slice assignment."""
    T = tnlib()
    rows, cols, depth, seed = 6, 6, 16, 2
    n = 36
    open_q = tuple(range(30, 36))
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=10, search_trials=64, seed=1)
    info = p.info()
    assert info["num_slices"] == 1024
    wires = p.sliced_wires()
    words = I.bitstrings(n, 4, seed)
    gates = OC.random_circuit(rows, cols, depth, seed)
    bits = I.bits_of(words[0], n)
    for s in (0, 777):
        got = p.contract_amplitudes(words[:1], slice_begin=s, slice_count=1)[0]
        fixed = {wires[j]: (s >> j) & 1 for j in range(len(wires))}
        ref = replay(p, gates, n, bits, open_q, fixed)
        assert rel(got, ref) <= 1e-5, s
        # the tensor-core path (bf16 hi+lo split, operand planes handed from
        # producer to consumer) on the same slice: the split-precision bound
        got = p.contract_amplitudes(words[:1], slice_begin=s, slice_count=1, precision="split_bf16")[0]
        assert rel(got, ref) <= 1e-4, s
        for mode in ("split_fp16", "scaled_fp16", "scaled_bf16"):
            got = p.contract_amplitudes(words[:1], slice_begin=s, slice_count=1, precision=mode)[0]
            assert rel(got, ref) <= MODE_BOUND[mode], (s, mode, rel(got, ref))


def test_full_size_6x6_bitstring_batch_vs_oracle():
    """The 6x6 benchmark plan on one slice for all four bitstrings of the batch
    at once: the bitstring-dependent steps run with the batch in the launch
    grid, and narrow tensor-core steps whose slice-only operand is shared by
    the bitstrings fold the bitstrings into the columns of one tile.  Every
    bitstring against the oracle, and the batch equal to the bitstrings one at
    a time."""
    T = tnlib()
    rows, cols, depth, seed = 6, 6, 16, 2
    n = 36
    open_q = tuple(range(30, 36))
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=10, search_trials=64, seed=1)
    wires = p.sliced_wires()
    words = I.bitstrings(n, 4, seed)
    gates = OC.random_circuit(rows, cols, depth, seed)
    s = 5
    fixed = {wires[j]: (s >> j) & 1 for j in range(len(wires))}
    got = p.contract_amplitudes(words, slice_begin=s, slice_count=1, precision="split_bf16")
    for b in range(4):
        ref = replay(p, gates, n, I.bits_of(words[b], n), open_q, fixed)
        assert rel(got[b], ref) <= 1e-4, b
        one = p.contract_amplitudes(words[b:b + 1], slice_begin=s, slice_count=1, precision="split_bf16")[0]
        assert rel(got[b], one) <= 1e-6, b


def test_split_bf16_path_vs_statevector():
    """A plan whose dense steps run on the tcgen05 kernel (bf16 hi+lo):
    relative L2 <= 1e-4 against the state vector."""
    T = tnlib()
    rows, cols, depth, seed, open_q = 4, 5, 14, 12, (14, 15, 16, 17, 18, 19)
    n = rows * cols
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=2, search_trials=32, seed=3)
    words = I.bitstrings(n, 3, seed)
    got, rep = p.contract_amplitudes(words, precision="split_bf16", report=True, profile=True)
    gates = OC.random_circuit(rows, cols, depth, seed)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in words], open_q)
    assert rel(got, ref) <= 1e-4
    c64 = p.contract_amplitudes(words, precision="c64")
    assert rel(c64, ref) <= 1e-5


MODE_BOUND = {"c64": 1e-5, "split_bf16": 1e-4, "split_fp16": 1e-4, "scaled_fp16": 2e-2, "scaled_bf16": 2e-2}


@pytest.mark.parametrize("mode", ["split_fp16", "scaled_fp16", "scaled_bf16"])
def test_scaled_and_split_fp16_modes_vs_statevector(mode):
    """Mixed-precision modes with per-unit power-of-two exponents on the
    tensor cores, against the state vector within each mode's bound."""
    T = tnlib()
    rows, cols, depth, seed, open_q = 4, 5, 14, 12, (14, 15, 16, 17, 18, 19)
    n = rows * cols
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=2, search_trials=32, seed=3)
    words = I.bitstrings(n, 3, seed)
    got, rep = p.contract_amplitudes(words, precision=mode, report=True)
    gates = OC.random_circuit(rows, cols, depth, seed)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in words], open_q)
    assert rel(got, ref) <= MODE_BOUND[mode], (mode, rel(got, ref))
    assert rep["discarded_units"] == 0


def test_filter_recompute_and_discard():
    """The filter of the scaled modes, driven by host-injected flags: a
    flagged unit is recomputed in complex64 (policy 0) or left out of the sum
    (policy 1, the paper's discard), which leaves the exact partial sum over
    the kept slices."""
    T = tnlib()
    rows, cols, depth, seed, open_q = 4, 4, 10, 5, (15, 14)
    n = rows * cols
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=4, search_trials=16, seed=3)
    words = I.bitstrings(n, 2, seed)
    base = p.contract_amplitudes(words, precision="scaled_fp16")
    got, rep = p.contract_amplitudes(words, precision="scaled_fp16", test_flag_every=3, report=True)
    flagged = [s for s in range(16) if s % 3 == 0]
    assert rep["flagged_units"] == len(flagged) * 2 and rep["discarded_units"] == 0
    assert rel(got, base) <= 2e-2
    got, rep = p.contract_amplitudes(words, precision="scaled_fp16", test_flag_every=3, overflow_policy=1,
                                     report=True)
    assert rep["discarded_units"] == len(flagged) * 2
    gates = OC.random_circuit(rows, cols, depth, seed)
    wires = p.sliced_wires()
    for bi, w in enumerate(words):
        net = OTN.circuit_network(gates, n, I.bits_of(w, n), open_q)
        ref = OTN.contract_sliced(net, wires, [s for s in range(16) if s not in flagged])
        assert rel(got[bi], ref) <= 2e-2


@pytest.mark.parametrize("mode", ["c64", "split_bf16", "scaled_fp16"])
def test_graph_replay_and_autotune_give_identical_sums(mode):
    """Batching: the per-group launch sequences replayed from CUDA graphs and
    the autotuned tensor-core tiles change neither the arithmetic nor its
    order, so the sums are bit-identical; several groups and a partial last
    group exercise graph reuse and the direct fallback."""
    T = tnlib()
    rows, cols, depth, seed, open_q = 4, 5, 14, 12, (14, 15, 16, 17, 18, 19)
    n = rows * cols
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=3, search_trials=32, seed=3)
    words = I.bitstrings(n, 3, seed)
    import torch
    s = torch.cuda.Stream()  # graphs need an explicit stream
    base = p.contract_amplitudes(words, precision=mode, units_per_group=3, stream=s)
    for _ in range(2):
        g = p.contract_amplitudes(words, precision=mode, units_per_group=3, use_graph=1, stream=s)
        assert np.array_equal(g, base)
    t = p.contract_amplitudes(words, precision=mode, units_per_group=3, autotune=1, stream=s)
    assert np.array_equal(t, base)
    t = p.contract_amplitudes(words, precision=mode, units_per_group=3, autotune=1, use_graph=1, stream=s)
    assert np.array_equal(t, base)
    # and every one of them is the right answer: the state vector
    gates = OC.random_circuit(rows, cols, depth, seed)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in words], open_q)
    assert rel(base, ref) <= {"c64": 1e-5, "split_bf16": 1e-4, "scaled_fp16": 2e-2}[mode]


@pytest.mark.parametrize("mode,tol", [("c64", 1e-5), ("split_fp16", 1e-4), ("scaled_bf16", 2e-2)])
def test_lattice_ordered_plan_vs_statevector(mode, tol):
    """A plan from the PEPS-style lattice sweep (order_generator=1; Sec. "A
    PEPS-based Simulation Method with an Optimized Slicing Strategy")
    contracted on the GPU, sliced and with open qubits, against the state
    vector."""
    T = tnlib()
    rows, cols, depth, seed, open_q = 4, 5, 12, 13, (15, 16, 17, 18, 19)
    n = rows * cols
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=4, search_trials=4, seed=1, order_generator=1)
    assert p.info()["num_sliced"] == 4
    words = I.bitstrings(n, 3, seed)
    got = p.contract_amplitudes(words, precision=mode)
    gates = OC.random_circuit(rows, cols, depth, seed)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in words], open_q)
    assert rel(got, ref) <= tol


@pytest.mark.parametrize("cap_aware", [0, 1])
def test_full_size_8x8_sampled_slices_vs_oracle(cap_aware):
    """8x8 grid (64 qubits), depth 1+20+1, seed 4, per-slice width capped at
    2^26, ten open qubits (1024 correlated amplitudes per bitstring): two
    sampled slices against the oracle's FP64 contraction of the same slice
    assignment, in complex64 and in split fp16; with the plain search and
    with width-cap-aware subtree rewrites (68 instead of 80 sliced indices)."""
    T = tnlib()
    rows, cols, depth, seed = 8, 8, 20, 4
    n = 64
    open_q = tuple(range(54, 64))
    p = _setup(T, rows, cols, depth, seed, open_q, max_log2_intermediate=26, search_trials=8 if not cap_aware else 16,
               seed=1, cap_aware_rewrites=cap_aware)
    info = p.info()
    assert info["max_log2_intermediate"] <= 26
    wires = p.sliced_wires()
    words = I.bitstrings(n, 1, seed)
    gates = OC.random_circuit(rows, cols, depth, seed)
    bits = I.bits_of(words[0], n)
    for s in (0, 4095):
        fixed = {wires[j]: (s >> j) & 1 for j in range(len(wires))}
        ref = replay(p, gates, n, bits, open_q, fixed)
        got = p.contract_amplitudes(words, slice_begin=s, slice_count=1)[0]
        assert got.shape == (1024,)
        assert rel(got, ref) <= 1e-5, s
        got = p.contract_amplitudes(words, slice_begin=s, slice_count=1, precision="split_fp16")[0]
        assert rel(got, ref) <= 1e-4, s


@pytest.fixture(scope="module")
def subcase_5x6():
    """The 30-qubit sub-case of the 6x6 workload: 5x6 grid, depth 1+16+1,
    circuit seed 2, the last 6 qubits open (64 amplitudes), 10 sliced indices
    (1024 slices), one bitstring of the seed-2 bitstring stream.  The FP64
    oracle sums every slice of the plan's tree."""
    T = tnlib()
    rows, cols, depth, seed = 5, 6, 16, 2
    n = rows * cols
    open_q = tuple(range(n - 6, n))
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=10, search_trials=32, seed=1,
               max_log2_intermediate=22)
    assert p.info()["num_slices"] == 1024
    words = I.bitstrings(n, 1, seed)
    gates = OC.random_circuit(rows, cols, depth, seed)
    wires = p.sliced_wires()
    bits = I.bits_of(words[0], n)
    ref = np.zeros(64, dtype=np.complex128)
    for s in range(1024):
        fixed = {wires[j]: (s >> j) & 1 for j in range(len(wires))}
        ref += replay(p, gates, n, bits, open_q, fixed)
    return p, words, ref


@pytest.mark.parametrize("mode", list(MODE_BOUND))
def test_30_qubit_subcase_every_mode_vs_fp64_oracle(subcase_5x6, mode):
    """All 1024 slices summed on the GPU, in each precision mode, against the
    oracle's exact FP64 sum, within the mode's bound."""
    p, words, ref = subcase_5x6
    got, rep = p.contract_amplitudes(words, precision=mode, report=True)
    assert rel(got[0], ref) <= MODE_BOUND[mode], (mode, rel(got[0], ref))
    assert rep["discarded_units"] == 0


@pytest.mark.parametrize("mode", list(MODE_BOUND))
def test_xeb_within_one_percent_of_the_oracle(mode):
    """Linear XEB of bitstrings drawn from the exact output distribution
    (state vector, inverse CDF of seeded uniforms), scored once with the
    oracle's probabilities and once with the GPU's: the two must agree within
    1% of the oracle's value.  The Porter-Thomas moments of the GPU's
    probabilities over the uniformly drawn bitstrings agree with the oracle's
    the same way."""
    from oracle import stats as ST
    T = tnlib()
    rows, cols, depth, seed = 4, 5, 14, 21
    n = rows * cols
    open_q = (16, 17, 18, 19)
    gates = OC.random_circuit(rows, cols, depth, seed)
    psi = SV.simulate(gates, n)
    p_all = np.abs(psi) ** 2
    u = np.random.default_rng(seed).random(400)
    idx = ST.sample_inverse_cdf(p_all, u)
    sample_bits = [[(int(i) >> q) & 1 for q in range(n)] for i in idx]
    words = np.stack([I.pack_bits(b) for b in sample_bits])
    plan = _setup(T, rows, cols, depth, seed, open_q, num_sliced=4, search_trials=32, seed=3)
    amps = plan.contract_amplitudes(words, precision=mode)
    col = [sum(b[q] << t for t, q in enumerate(open_q)) for b in sample_bits]
    p_gpu = np.abs(amps[np.arange(len(idx)), col]) ** 2
    f_ref = ST.linear_xeb(p_all[idx], n)
    f_gpu = ST.linear_xeb(p_gpu, n)
    assert f_ref > 0.5
    assert abs(f_gpu - f_ref) <= 0.01 * abs(f_ref), (mode, f_gpu, f_ref)
    uni = I.bitstrings(n, 64, seed)
    ref_u = SV.amplitudes(psi, n, [I.bits_of(w, n) for w in uni], open_q)
    got_u = plan.contract_amplitudes(uni, precision=mode)
    m_ref = ST.porter_thomas_moments(np.abs(ref_u.ravel()) ** 2, n)
    m_gpu = ST.porter_thomas_moments(np.abs(got_u.ravel()) ** 2, n)
    assert np.allclose(m_gpu, m_ref, rtol=1e-2), (mode, m_gpu, m_ref)


def test_empty_batches_and_split_slice_ranges():
    """Edge cases of the call: no bitstrings, an empty slice range, and a sum
    split into two slice ranges (equal to the whole range up to the FP64
    rounding of one extra addition)."""
    T = tnlib()
    rows, cols, depth, seed, open_q = 4, 4, 10, 5, (15, 14)
    n = rows * cols
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=4, search_trials=16, seed=3)
    words = I.bitstrings(n, 3, seed)
    none = p.contract_amplitudes(words[:0])
    assert none.shape == (0, 4)
    zero = p.contract_amplitudes(words, slice_count=0)
    assert zero.shape == (3, 4) and not np.any(zero)
    for mode in ("c64", "split_bf16"):
        full = p.contract_amplitudes(words, precision=mode)
        a = p.contract_amplitudes(words, precision=mode, slice_begin=0, slice_count=7)
        b = p.contract_amplitudes(words, precision=mode, slice_begin=7)
        assert np.allclose(a + b, full, rtol=1e-12, atol=1e-15 * np.abs(full).max())
    with pytest.raises(T.TnError):
        p.contract_amplitudes(words, slice_begin=10, slice_count=7)


def test_autotune_choices_persist_in_the_cache_file(tmp_path, monkeypatch):
    """TN_AUTOTUNE_CACHE: the first plan that tunes writes its tile choices;
    a fresh plan of the same circuit reads them instead of tuning again, and
    every choice gives the same sums."""
    T = tnlib()
    import torch
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("TN_AUTOTUNE_CACHE", str(cache))
    rows, cols, depth, seed, open_q = 4, 5, 14, 12, (14, 15, 16, 17, 18, 19)
    n = rows * cols
    words = I.bitstrings(n, 3, seed)
    s = torch.cuda.Stream()
    p1 = _setup(T, rows, cols, depth, seed, open_q, num_sliced=3, search_trials=32, seed=3)
    base = p1.contract_amplitudes(words, precision="split_bf16", stream=s)
    t1 = p1.contract_amplitudes(words, precision="split_bf16", autotune=1, stream=s)
    assert np.array_equal(t1, base)
    lines = cache.read_text().split()
    assert len(lines) >= 6 and lines[0] == format(p1.info()["hash"], "x")
    p2 = _setup(T, rows, cols, depth, seed, open_q, num_sliced=3, search_trials=32, seed=3)
    t2 = p2.contract_amplitudes(words, precision="split_bf16", autotune=1, stream=s)
    assert np.array_equal(t2, base)
    assert cache.read_text().split() == lines  # read, not tuned again


def test_select_plan_keeps_the_fastest_probe_and_its_amplitudes():
    """Measured plan choice: every candidate is timed on the same probe, the
    one with the shortest time per slice is returned, and its amplitudes over
    all slices match the state vector."""
    T = tnlib()
    rows, cols, depth, seed, open_q = 4, 5, 14, 12, (16, 17, 18, 19)
    n = rows * cols
    net = T.build_network(T.random_circuit(rows, cols, depth, seed), list(open_q))
    words = I.bitstrings(n, 2, seed)
    best, table = T.select_plan(net, words, seeds=(1, 2, 3), probe_slices=8, precision="c64", num_sliced=5,
                                search_trials=16)
    assert len(table) == 3
    fastest = min(table, key=lambda r: r[1])
    assert best.info()["hash"] == fastest[2]
    got = best.contract_amplitudes(words)
    gates = OC.random_circuit(rows, cols, depth, seed)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in words], open_q)
    assert rel(got, ref) <= 1e-5


def test_graphs_follow_buffer_and_handover_changes():
    """Replayed launch sequences hold buffer addresses: a call that needs
    larger arenas (more bitstrings) replaces the buffers and the recorded
    sequences with them, and the plane handover is part of a sequence's key.
    Every graph-replayed result equals the direct launches."""
    T = tnlib()
    import torch
    rows, cols, depth, seed, open_q = 4, 5, 14, 12, (14, 15, 16, 17, 18, 19)
    n = rows * cols
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=3, search_trials=32, seed=3)
    s = torch.cuda.Stream()
    for nb in (1, 3, 1, 2, 3, 1):
        words = I.bitstrings(n, nb, seed + nb)
        base = p.contract_amplitudes(words, precision="split_bf16", units_per_group=3, stream=s)
        g = p.contract_amplitudes(words, precision="split_bf16", units_per_group=3, use_graph=1, stream=s)
        assert np.array_equal(g, base), nb
    words = I.bitstrings(n, 2, seed)
    for ho in (1, 2, 1, 2):
        base = p.contract_amplitudes(words, precision="scaled_fp16", handover=ho, stream=s)
        g = p.contract_amplitudes(words, precision="scaled_fp16", handover=ho, use_graph=1, stream=s)
        assert np.array_equal(g, base), ho


def test_failed_device_allocations_report_errors_and_recover(monkeypatch):
    """Host-side fault injection (TN_FAULT_ALLOC=k fails the executor's k-th
    device allocation): every failure point returns an error status instead
    of crashing, and the same plan then contracts correctly once allocations
    succeed again."""
    T = tnlib()
    rows, cols, depth, seed, open_q = 4, 4, 10, 5, (15, 14)
    n = rows * cols
    words = I.bitstrings(n, 2, seed)
    gates = OC.random_circuit(rows, cols, depth, seed)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in words], open_q)
    failures = 0
    for k in range(1, 25):
        p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=4, search_trials=16, seed=3)
        monkeypatch.setenv("TN_FAULT_ALLOC", f"{k}")
        try:
            p.contract_amplitudes(words, precision="split_bf16")
        except T.TnError as e:
            assert e.status in (3, 4), e   # TN_EHBM or TN_ECUDA
            failures += 1
        monkeypatch.delenv("TN_FAULT_ALLOC")
        got = p.contract_amplitudes(words, precision="split_bf16")
        assert rel(got, ref) <= 1e-4, k
    assert failures >= 8


def test_precision_analysis_keeps_the_sensitive_steps_accurate():
    """Per-step precision from a pre-analysis (Sec. "A Mixed-Precision
    Computation Method via Adaptive Precision Scaling"): on a probe of four
    slices the analysis keeps the most error-sensitive steps in split fp16 and
    the rest in scaled bf16.  The mixed assignment meets the target on the
    probe, keeps only part of the steps accurate, and over all slices lands
    between the all-accurate and the all-fast errors against the state vector."""
    T = tnlib()
    rows, cols, depth, seed, open_q = 4, 5, 16, 2, (14, 15, 16, 17, 18, 19)
    n = rows * cols
    p = _setup(T, rows, cols, depth, seed, open_q, num_sliced=6, search_trials=16, seed=1)
    words = I.bitstrings(n, 2, seed)
    # a target every step meets: nothing kept accurate
    sp0, rep0 = p.precision_analysis(words[:1], probe_slices=4, fast="scaled_bf16", accurate="split_fp16",
                                     target=1.0)
    assert rep0["accurate_steps"] == 0 and (sp0 != 2).all() and rep0["candidate_steps"] > 1, rep0
    assert rep0["err_fast"] > 1e-3 and rep0["err_accurate"] <= 1e-4, rep0
    # half the all-fast error: the most sensitive steps, not all of them
    target = rep0["err_fast"] / 2
    sp, rep = p.precision_analysis(words[:1], probe_slices=4, fast="scaled_bf16", accurate="split_fp16",
                                   target=target)
    assert rep["err_mixed"] <= target and 0 < rep["accurate_steps"] < rep["candidate_steps"], rep
    assert set(np.unique(sp)) <= {-1, 2, 4}
    assert int((sp == 2).sum()) == rep["accurate_steps"]
    gates = OC.random_circuit(rows, cols, depth, seed)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in words], open_q)
    mixed = rel(p.contract_amplitudes(words, precision="c64", step_precision=sp), ref)
    fast = rel(p.contract_amplitudes(words, precision="scaled_bf16"), ref)
    accurate = rel(p.contract_amplitudes(words, precision="split_fp16"), ref)
    assert accurate <= 1e-4 and mixed < 0.8 * fast, (accurate, mixed, fast)


@pytest.mark.parametrize("mode,tol", [("c64", 1e-5), ("split_fp16", 1e-4)])
def test_split_diagonal_plan_vs_statevector(mode, tol):
    """The network with every fSim(pi/2, pi/6) turned into a wire swap plus a
    rank-2 bond (TN_NET_SPLIT_DIAGONAL; Sec. "A PEPS-based Simulation Method
    with an Optimized Slicing Strategy", diagonal gates), planned with four
    sliced indices and five open qubits, contracted on the GPU."""
    T = tnlib()
    rows, cols, depth, seed, open_q = 4, 5, 12, 14, (15, 16, 17, 18, 19)
    n = rows * cols
    net = T.build_network(T.random_circuit(rows, cols, depth, seed), list(open_q), split_diagonal=True)
    p = T.plan(net, num_sliced=4, search_trials=16, seed=1)
    words = I.bitstrings(n, 3, seed)
    got = p.contract_amplitudes(words, precision=mode)
    gates = OC.random_circuit(rows, cols, depth, seed)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in words], open_q)
    assert rel(got, ref) <= tol


def test_split_diagonal_6x6_sampled_slice_vs_oracle():
    """The 6x6 workload's circuit (depth 1+16+1, seed 2, six open qubits) with
    split diagonals and 10 sliced indices: one sampled slice contracted on the
    GPU in complex64 against the oracle's hyperedge network (oracle.hyper)
    with the same index values, contracted in FP64 in the plan's order."""
    T = tnlib()
    from _replay import replay
    rows, cols, depth, seed = 6, 6, 16, 2
    n = 36
    open_q = tuple(range(30, 36))
    net = T.build_network(T.random_circuit(rows, cols, depth, seed), list(open_q), split_diagonal=True)
    p = T.plan(net, num_sliced=10, search_trials=64, seed=1)
    words = I.bitstrings(n, 1, seed)
    s = 613
    got = p.contract_amplitudes(words, precision="c64", slice_begin=s, slice_count=1)[0]
    wires = p.sliced_wires()
    gates = OC.random_circuit(rows, cols, depth, seed)
    ref = replay(p, gates, n, I.bits_of(words[0], n), open_q, {w: (s >> j) & 1 for j, w in enumerate(wires)},
                 split=True)
    assert rel(got, ref) <= 1e-5


def test_c_program_contracts_and_serves_through_the_abi(tmp_path):
    """A plain C99 program (tests/c_abi_contract.c) linked against the library
    calls tn_contract_amplitudes with host buffers in complex64 and split fp16
    and serves one request; its printed amplitudes match the state vector."""
    import os
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if not gcc:
        pytest.skip("no C compiler")
    T = tnlib()
    from paper_2110_14502_gb300 import _abi
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(_abi.LIB_PATH)
    exe = str(tmp_path / "c_abi_contract")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(root, "include"),
                    os.path.join(root, "tests", "c_abi_contract.c"), "-o", exe, "-L", libdir, "-ltn",
                    f"-Wl,-rpath,{libdir}"], check=True, capture_output=True, text=True)
    rows, cols, depth, seed, k = 4, 5, 12, 15, 3
    n = rows * cols
    words = I.bitstrings(n, 3, seed)
    r = subprocess.run([exe] + [f"{int(w):x}" for w in words.reshape(-1)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    got = {}
    for line in r.stdout.split("\n"):
        if line:
            tag, b, j, re_, im_ = line.split()
            got.setdefault(tag, np.zeros((len(words), 1 << k), dtype=np.complex128))[int(b), int(j)] = \
                float(re_) + 1j * float(im_)
    gates = OC.random_circuit(rows, cols, depth, seed)
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in words], tuple(range(n - k, n)))
    assert rel(got["c64"], ref) <= 1e-5 and rel(got["served"], ref) <= 1e-5
    assert rel(got["split_fp16"], ref) <= 1e-4
