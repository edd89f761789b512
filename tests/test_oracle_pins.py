"""Pins of the CPU oracle against facts it does not compute itself:
published generator outputs, closed-form gate identities, brute-force
Kronecker products, normalisation, exact slicing and order independence."""
import itertools

import numpy as np
import pytest

import tn_inputs as I
from oracle import circuit as C
from oracle import gates as G
from oracle import statevector as SV
from oracle import tn as TN

X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)


# ---- SplitMix64: published outputs (tests/golden/splitmix64.txt, with its citation)
def _golden_splitmix64():
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                seed, *outs = line.split()
                rows.append((int(seed, 0), [int(x, 0) for x in outs]))
    return rows


@pytest.mark.parametrize("cls", [I.SplitMix64, C._SplitMix64])
def test_splitmix64_published_vectors(cls):
    rows = _golden_splitmix64()
    assert len(rows) == 2
    for seed, outs in rows:
        r = cls(seed)
        assert [r.next() for _ in range(len(outs))] == outs


# ---- gate matrices
@pytest.mark.parametrize("U", [G.SQRT_X, G.SQRT_Y, G.SQRT_W, G.fsim(G.FSIM_THETA, G.FSIM_PHI), G.fsim(0.3, 1.1)])
def test_gates_unitary(U):
    assert np.allclose(U.conj().T @ U, np.eye(len(U)), atol=1e-15)


def test_sqrt_gates_square_to_minus_i_pauli():
    W = (X + Y) / np.sqrt(2)
    assert np.allclose(G.SQRT_X @ G.SQRT_X, -1j * X, atol=1e-15)
    assert np.allclose(G.SQRT_Y @ G.SQRT_Y, -1j * Y, atol=1e-15)
    assert np.allclose(G.SQRT_W @ G.SQRT_W, -1j * W, atol=1e-15)


def test_fsim_special_cases():
    assert np.allclose(G.fsim(0.0, 0.0), np.eye(4))
    F = G.fsim(np.pi / 2, 0.0)
    e01 = np.array([0, 1, 0, 0], dtype=complex)   # |x_a=0, x_b=1>
    assert np.allclose(F @ e01, [0, 0, -1j, 0])   # -> -i |10>
    F = G.fsim(np.pi / 2, np.pi / 6)
    assert np.isclose(F[3, 3], np.exp(-1j * np.pi / 6))
    assert np.isclose(F[0, 0], 1.0)


# ---- circuit protocol
def test_coupler_patterns_by_hand():
    # 3 x 4 grid, qubit (r, c) = 4r + c
    assert C.coupler_pattern(3, 4, 0) == [(0, 1), (2, 3), (4, 5), (6, 7), (8, 9), (10, 11)]
    assert C.coupler_pattern(3, 4, 1) == [(1, 2), (5, 6), (9, 10)]
    assert C.coupler_pattern(3, 4, 2) == [(0, 4), (1, 5), (2, 6), (3, 7)]
    assert C.coupler_pattern(3, 4, 3) == [(4, 8), (5, 9), (6, 10), (7, 11)]
    # every grid edge appears in exactly one pattern
    edges = set()
    for p in range(4):
        for e in C.coupler_pattern(5, 6, p):
            assert e not in edges
            edges.add(e)
    assert len(edges) == 5 * 5 + 4 * 6


def test_circuit_layout_and_no_repeat():
    rows, cols, depth = 3, 4, 9
    n = rows * cols
    gs = C.random_circuit(rows, cols, depth, seed=7)
    n_fsim = sum(len(C.coupler_pattern(rows, cols, c % 4)) for c in range(depth))
    assert len(gs) == n * (depth + 1) + n_fsim
    last = {}
    for g in gs:
        if len(g.qubits) == 1:
            q = g.qubits[0]
            assert last.get(q) != g.kind
            last[q] = g.kind
        else:
            assert g.kind == "fsim" and g.qubits[0] < g.qubits[1]


def test_circuit_draws_follow_splitmix64():
    """Layer 0 kinds are KINDS[((x >> 32) * 3) >> 32] of the published stream,
    layer 1 picks among the two other kinds with ((x >> 32) * 2) >> 32."""
    rows, cols = 2, 3
    n = rows * cols
    gs = C.random_circuit(rows, cols, 1, seed=1234567)
    r = I.SplitMix64(1234567)
    first = [G.ONE_QUBIT_KINDS[((r.next() >> 32) * 3) >> 32] for _ in range(n)]
    assert [g.kind for g in gs[:n]] == first
    second = []
    for q in range(n):
        opts = [k for k in G.ONE_QUBIT_KINDS if k != first[q]]
        second.append(opts[((r.next() >> 32) * 2) >> 32])
    assert [g.kind for g in gs if len(g.qubits) == 1][n:] == second


# ---- state vector
def _kron_unitary(gates, n):
    """Dense 2^n x 2^n unitary by Kronecker products (qubit 0 = LSB)."""
    I2 = np.eye(2)
    U = np.eye(1 << n, dtype=complex)
    for g in gates:
        if len(g.qubits) == 1:
            q = g.qubits[0]
            M = np.array([[1.0]])
            for k in reversed(range(n)):
                M = np.kron(M, g.matrix if k == q else I2)
        else:
            a, b = g.qubits
            M = np.zeros((1 << n, 1 << n), dtype=complex)
            for i in range(1 << n):
                xa, xb = (i >> a) & 1, (i >> b) & 1
                for ya, yb in itertools.product((0, 1), repeat=2):
                    j = i & ~(1 << a) & ~(1 << b) | (ya << a) | (yb << b)
                    M[j, i] += g.matrix[2 * ya + yb, 2 * xa + xb]
        U = M @ U
    return U


@pytest.mark.parametrize("rows,cols,depth,seed", [(1, 2, 3, 1), (2, 2, 4, 2), (1, 4, 5, 3), (2, 2, 8, 4)])
def test_statevector_matches_kronecker(rows, cols, depth, seed):
    n = rows * cols
    gs = C.random_circuit(rows, cols, depth, seed)
    psi = SV.simulate(gs, n)
    U = _kron_unitary(gs, n)
    assert np.allclose(psi, U[:, 0], atol=1e-13)


def test_statevector_hand_cases():
    # sqrt(X)|0> = (|0> - i|1>)/sqrt2
    g = C.Gate("sqrtx", (0,), matrix=G.SQRT_X)
    psi = SV.simulate([g], 1)
    assert np.allclose(psi, np.array([1, -1j]) / np.sqrt(2))
    # fSim(pi/2, 0) on qubits (0, 1): |x0=0, x1=1> -> -i |x0=1, x1=0>
    flip1 = C.Gate("mat1", (1,), matrix=X)
    fs = C.Gate("fsim", (0, 1), np.pi / 2, 0.0, G.fsim(np.pi / 2, 0.0))
    psi = SV.simulate([flip1, fs], 2)
    assert np.allclose(psi, [0, -1j, 0, 0])   # index 1 = qubit 0 set


@pytest.mark.parametrize("rows,cols,depth", [(3, 3, 8), (3, 4, 10)])
def test_statevector_norm(rows, cols, depth):
    psi = SV.simulate(C.random_circuit(rows, cols, depth, 5), rows * cols)
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-12


def test_amplitude_open_index_convention():
    n = 3
    psi = np.arange(8, dtype=complex)
    a = SV.amplitudes(psi, n, [[1, 0, 0]], open_qubits=(2, 1))
    # j bit0 -> qubit 2, bit1 -> qubit 1; qubit 0 fixed to 1
    assert list(a[0].real) == [1, 5, 3, 7]


# ---- tensor network
def _rows(n, nb, seed):
    return [I.bits_of(w, n) for w in I.bitstrings(n, nb, seed)]


@pytest.mark.parametrize("rows,cols,depth,seed,opened", [(3, 3, 6, 1, ()), (3, 4, 8, 2, (10, 11)), (2, 5, 10, 3, (0, 9, 4))])
def test_tn_matches_statevector(rows, cols, depth, seed, opened):
    n = rows * cols
    gs = C.random_circuit(rows, cols, depth, seed)
    bits = _rows(n, 3, seed)
    a_sv = SV.amplitudes(SV.simulate(gs, n), n, bits, opened)
    a_tn = TN.amplitudes(gs, n, bits, opened)
    assert np.linalg.norm(a_tn - a_sv) / np.linalg.norm(a_sv) < 1e-12


def _random_tree(labels, seed):
    """A random contraction tree that only joins tensors sharing an index
    (random outer products of many tensors would blow up memory)."""
    rng = np.random.default_rng(seed)
    active = {i: set(l) for i, l in enumerate(labels)}
    nid = len(labels)
    pairs = []
    while len(active) > 1:
        keys = sorted(active)
        cand = [(a, b) for x, a in enumerate(keys) for b in keys[x + 1:] if active[a] & active[b]]
        if not cand:
            cand = [(keys[0], keys[1])]
        a, b = cand[rng.integers(len(cand))]
        active[nid] = active.pop(a) ^ active.pop(b)
        pairs.append((a, b))
        nid += 1
    return pairs


def test_tn_order_independence():
    rows, cols, depth = 2, 3, 6
    n = rows * cols
    gs = C.random_circuit(rows, cols, depth, 11)
    net = TN.circuit_network(gs, n, _rows(n, 1, 11)[0], open_qubits=(5,))
    ref = TN.contract(net)
    for s in range(3):
        v = TN.contract(net, _random_tree(net.labels, s))
        assert np.linalg.norm(v - ref) <= 1e-12 * np.linalg.norm(ref)


def test_tn_sliced_sum_equals_unsliced():
    rows, cols, depth = 3, 3, 8
    n = rows * cols
    gs = C.random_circuit(rows, cols, depth, 13)
    net = TN.circuit_network(gs, n, _rows(n, 1, 13)[0], open_qubits=(8,))
    ref = TN.contract(net)
    internal = sorted({l for ls in net.labels for l in ls} - set(net.open_labels))
    rng = np.random.default_rng(0)
    sliced = [internal[i] for i in rng.choice(len(internal), 5, replace=False)]
    tot = TN.contract_sliced(net, sliced)
    assert np.linalg.norm(tot - ref) <= 1e-12 * np.linalg.norm(ref)
    # one slice is the contraction with those wires fixed, brute force:
    s = 19
    fixed = TN.fix_indices(net, {lab: (s >> j) & 1 for j, lab in enumerate(sliced)})
    assert np.allclose(TN.contract_slice(net, sliced, s), TN.contract(fixed))


# ---- work count of a contraction tree (oracle.replay.work_cmac): the complex
# multiply-adds of the pairwise steps between leaf groups, 2^|A u B| each
# (Sec. "How Performance Was Measured": count the arithmetic performed).

def _gate(kind, qubits):
    mats = {"sqrtx": G.SQRT_X, "sqrty": G.SQRT_Y, "sqrtw": G.SQRT_W}
    if kind == "fsim":
        return C.Gate("fsim", qubits, G.FSIM_THETA, G.FSIM_PHI, G.fsim(G.FSIM_THETA, G.FSIM_PHI))
    return C.Gate(kind, qubits, matrix=mats[kind])


def test_work_cmac_hand_counts():
    from oracle.replay import work_cmac
    # one qubit, X then Y then W, raw ids 0..2 the gates and 3 the |0> input:
    # <x| W Y X |0> is two 2x2 matrix-vector products (4 MACs each) and one
    # length-2 dot product with the projector folded into W's group (2 MACs)
    g1 = [_gate("sqrtx", (0,)), _gate("sqrty", (0,)), _gate("sqrtw", (0,))]
    groups = [[3], [0], [1], [2]]
    pairs = [(0, 1), (4, 2), (5, 3)]
    assert work_cmac(g1, 1, [1], [], groups, pairs) == 10.0
    # the same with the qubit open: no projector, the last step is a 2x2
    # matrix-vector product (4 MACs)
    assert work_cmac(g1, 1, [0], [0], groups, pairs) == 12.0
    # two qubits, X on 0 then fSim(0, 1): each input meets its neighbour (4 +
    # 4 MACs), the two rank-1 results meet in a dot product (2 MACs); fSim's
    # group absorbs both projectors
    g2 = [_gate("sqrtx", (0,)), _gate("fsim", (0, 1))]
    assert work_cmac(g2, 2, [0, 1], [], [[2], [3], [0], [1]], [(0, 2), (1, 3), (4, 5)]) == 10.0
    # merging the |0> of qubit 0 into the X group moves that product inside a
    # leaf group, where it is not counted: 4 + 2 MACs remain
    assert work_cmac(g2, 2, [0, 1], [], [[2, 0], [3], [1]], [(1, 2), (0, 3)]) == 6.0


def test_work_cmac_equals_the_products_of_the_actual_contraction():
    """On random small circuits and random trees over single-tensor groups,
    the count equals the sum over the tensordot calls of the oracle's own
    contraction of (elements of A) x (elements of B) / (contracted extent)."""
    from oracle.replay import work_cmac
    for seed in range(4):
        rows, cols, depth = 2, 2 + seed % 2, 3 + seed
        gates = C.random_circuit(rows, cols, depth, seed)
        n = rows * cols
        bits = [int(b) for b in _rows(n, 1, seed)[0]]
        open_q = [n - 1] if seed % 2 else []
        net = TN.circuit_network(gates, n, bits, open_q)
        ng = len(gates)
        closed = [q for q in range(n) if q not in open_q]
        last = {q: ng + q for q in range(n)}
        for gi, g in enumerate(gates):
            for q in g.qubits:
                last[q] = gi
        # raw id r (gate or input) -> network tensors of its group (+ projectors)
        raws = list(range(ng)) + [ng + q for q in range(n)]
        groups = [[r] for r in raws]
        members = []
        for r in raws:
            m = [r + n if r < ng else r - ng]
            m += [n + ng + i for i, q in enumerate(closed) if last[q] == r]
            members.append(m)
        tens, labs = [], []
        for m in members:
            t, l = net.tensors[m[0]], list(net.labels[m[0]])
            for i in m[1:]:
                t, l = _contract_counted(t, l, net.tensors[i], list(net.labels[i]), [0])
            tens.append(t)
            labs.append(l)
        rng = np.random.default_rng(seed)
        live, pairs, nid, work = list(range(len(tens))), [], len(tens), [0]
        store = dict(enumerate(zip(tens, labs)))
        while len(live) > 1:
            # a random live tensor and a random partner sharing an index with
            # it (any partner once the network has become disconnected)
            i = int(rng.choice(live))
            nbr = [x for x in live if x != i and set(store[x][1]) & set(store[i][1])]
            j = int(rng.choice(nbr if nbr else [x for x in live if x != i]))
            live.remove(i)
            live.remove(j)
            (ta, la), (tb, lb) = store.pop(i), store.pop(j)
            store[nid] = _contract_counted(ta, la, tb, lb, work)
            pairs.append((i, j))
            live.append(nid)
            nid += 1
        assert work_cmac(gates, n, bits, open_q, groups, pairs) == float(work[0]), seed


def _contract_counted(ta, la, tb, lb, work):
    shared = [x for x in la if x in lb]
    ia = [la.index(x) for x in shared]
    ib = [lb.index(x) for x in shared]
    work[0] += ta.size * tb.size // (2 ** len(shared))
    t = np.tensordot(ta, tb, axes=(ia, ib))
    return t, [x for x in la if x not in shared] + [x for x in lb if x not in shared]


# ---- hyperedge networks and the diagonal decomposition (oracle.hyper)

@pytest.mark.parametrize("phi", [np.pi / 6, 0.3, np.pi])
def test_fsim_half_pi_is_a_swap_times_its_diagonal(phi):
    """fSim(pi/2, phi) = SWAP diag(1, -i, -i, e^{-i phi}): the factors U
    (copy) and V (D) joined by the bond rebuild the gate exactly."""
    from oracle import hyper as H
    F = G.fsim(np.pi / 2, phi)
    D = H.swap_diagonal(F)
    assert np.allclose(D, [[1, -1j], [-1j, np.exp(-1j * phi)]], atol=1e-15)
    U, V = np.eye(2), D.T                                   # U[x_a, c], V[x_b, c]
    T = np.zeros((2, 2, 2, 2), dtype=np.complex128)         # [a', b', a, b]
    for a in range(2):
        for b in range(2):
            T[b, a, a, b] = sum(U[a, c] * V[b, c] for c in range(2))
    assert np.allclose(T.reshape(4, 4), F, atol=1e-15)


def test_swap_diagonal_rejects_other_gates():
    from oracle import hyper as H
    assert H.swap_diagonal(G.fsim(np.pi / 3, np.pi / 6)) is None
    assert H.swap_diagonal(np.kron(G.SQRT_X, np.eye(2))) is None
    assert H.swap_diagonal(np.diag([1, 1j, 1j, -1])) is None          # diagonal without the swap


def test_hyperedge_contraction_by_hand():
    """Three tensors on one index (a hyperedge): the first pair keeps the
    index for the third, which sums it: sum_x a_x M_xy c_x, by brute force."""
    from oracle import hyper as H
    rng = np.random.default_rng(5)
    a = rng.normal(size=2) + 1j * rng.normal(size=2)
    M = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    c = rng.normal(size=2) + 1j * rng.normal(size=2)
    want = np.array([sum(a[x] * M[x, y] * c[x] for x in range(2)) for y in range(2)])
    for pairs in ([(0, 1), (3, 2)], [(1, 2), (3, 0)], [(0, 2), (3, 1)]):
        t, l = H.contract_tree([a, M, c], [("x",), ("x", "y"), ("x",)], ["y"], pairs)
        assert l == ("y",) and np.allclose(t, want, atol=1e-14), pairs


@pytest.mark.parametrize("rows,cols,depth,seed,opened", [(3, 3, 6, 1, ()), (2, 4, 8, 2, (6, 7)), (3, 4, 6, 3, (0, 11))])
def test_split_network_matches_statevector(rows, cols, depth, seed, opened):
    from oracle import hyper as H
    gates = C.random_circuit(rows, cols, depth, seed)
    n = rows * cols
    rows_ = _rows(n, 2, seed)
    psi = SV.simulate(gates, n)
    ref = SV.amplitudes(psi, n, rows_, opened)
    got = H.amplitudes(gates, n, rows_, opened)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    # every fSim of the benchmark gate set was decomposed: no rank-4 tensor left
    net = H.circuit_network_split(gates, n, rows_[0], opened)
    assert max(len(l) for l in net.labels) == 2


def test_split_network_sliced_sum_equals_unsliced():
    """Slicing a hyperedge wire index fixes it in all three holders; slicing
    a bond fixes it in both factors; the sum over assignments is unchanged."""
    from oracle import hyper as H
    gates = C.random_circuit(3, 3, 8, 4)
    n = 9
    bits = _rows(n, 1, 4)
    net = H.circuit_network_split(gates, n, bits[0], (8,))
    count = {}
    for ls in net.labels:
        for x in ls:
            count[x] = count.get(x, 0) + 1
    hyper_wires = [x for x, k in count.items() if k == 3][:2]
    bonds = [x for x in count if x[0] < 0][:2]
    assert len(hyper_wires) == 2 and len(bonds) == 2
    full = H.amplitudes(gates, n, bits, (8,))
    sliced = H.amplitudes(gates, n, bits, (8,), sliced=hyper_wires + bonds)
    assert np.linalg.norm(sliced - full) <= 1e-12 * np.linalg.norm(full)
