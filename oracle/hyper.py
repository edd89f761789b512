"""Hyperedge tensor networks and the diagonal decomposition of swap-like gates.

Test infrastructure: only the test suite may import this module; the library
shares no code with it.  Plain NumPy, complex128.

fSim(pi/2, phi) maps |x_a x_b> to D(x_a, x_b) |x_b x_a> with D the diagonal
diag(1, -i, -i, e^{-i phi}) in the basis 2 x_a + x_b: a wire swap times a
diagonal gate.  Sec. "A PEPS-based Simulation Method with an Optimized
Slicing Strategy" treats the indices of diagonal gates as hyperedges.  In
the network built here such a gate has no tensor of its own:

* the swap renames the wires: the index on qubit a's wire before the gate
  continues as qubit b's wire after it, and vice versa;
* the diagonal has operator-Schmidt rank 2,
      D(x, y) = sum_c delta(x, c) D(c, y),
  so it becomes two factors joined by a bond index c of dimension 2:
      U_g(x_a, c) = delta(x_a, c),     V_g(x_b, c) = D(c, x_b).

A wire index is then held by three tensors (the tensor that produced it, a
factor, and the next tensor on the swapped wire): a hyperedge.  A pairwise
contraction therefore sums a shared index only when no other tensor and no
open output still holds it; otherwise the index stays in the product (a
batch index), which ``numpy.einsum`` with explicit output subscripts states
directly.  Fixing an index (slicing) fixes it in every holder.

Index names follow ``oracle.tn``: ``(q, t)`` is qubit q's wire after its t-th
one-qubit (or unsplit two-qubit) gate; the bond of gate g is ``(-1 - g, 0)``.
Every tensor records the raw id it came from: gate g -> g, the |0> input of
qubit q -> num_gates + q, the factors of gate g -> num_gates + n + 2g (U) and
+ 1 (V), the projector <x_q| of a closed qubit -> -(q + 1).
"""
from collections import defaultdict

import numpy as np

from . import tn as OTN


def swap_diagonal(matrix):
    """D (2x2, D[x, y] = factor of |x_a = x, x_b = y>) when the 4x4 gate
    (basis 2 x_a + x_b, rows = outputs) is a wire swap times a diagonal,
    else None."""
    m = np.asarray(matrix, dtype=np.complex128).reshape(4, 4)
    swap_of = [0, 2, 1, 3]  # column 2 x_a + x_b  ->  row 2 x_b + x_a
    off = sum(abs(m[r, c]) for r in range(4) for c in range(4) if r != swap_of[c])
    if off > 1e-12:
        return None
    D = np.zeros((2, 2), dtype=np.complex128)
    for x in range(2):
        for y in range(2):
            D[x, y] = m[2 * y + x, 2 * x + y]
    return D


class HyperNetwork:
    def __init__(self, tensors, labels, open_labels, raw):
        self.tensors = list(tensors)
        self.labels = [tuple(l) for l in labels]
        self.open_labels = list(open_labels)
        self.raw = list(raw)


def circuit_network_split(gates, n, bits=None, open_qubits=()):
    """Network of <x|U|0^n> with every swap-times-diagonal two-qubit gate
    decomposed as described above (other gates as in ``oracle.tn``)."""
    open_qubits = list(open_qubits)
    ng = len(gates)
    seg = [0] * n
    cur = [(q, 0) for q in range(n)]
    producer = {}  # wire index -> raw id of the tensor that created it
    tensors, labels, raw = [], [], []
    for q in range(n):
        tensors.append(np.array([1.0, 0.0], dtype=np.complex128))
        labels.append((cur[q],))
        raw.append(ng + q)
        producer[cur[q]] = ng + q
    for g, gate in enumerate(gates):
        if len(gate.qubits) == 1:
            (q,) = gate.qubits
            w_in = cur[q]
            seg[q] += 1
            cur[q] = (q, seg[q])
            tensors.append(np.array(gate.matrix, dtype=np.complex128))      # [out, in]
            labels.append((cur[q], w_in))
            raw.append(g)
            producer[cur[q]] = g
            continue
        a, b = gate.qubits
        D = swap_diagonal(gate.matrix)
        if D is None:
            ia, ib = cur[a], cur[b]
            seg[a] += 1
            seg[b] += 1
            cur[a], cur[b] = (a, seg[a]), (b, seg[b])
            tensors.append(np.array(gate.matrix, dtype=np.complex128).reshape(2, 2, 2, 2))
            labels.append((cur[a], cur[b], ia, ib))
            raw.append(g)
            producer[cur[a]] = producer[cur[b]] = g
            continue
        xa, xb, bond = cur[a], cur[b], (-1 - g, 0)
        tensors.append(np.eye(2, dtype=np.complex128))                  # U[x_a, c] = delta
        labels.append((xa, bond))
        raw.append(ng + n + 2 * g)
        tensors.append(D.T.copy())                                      # V[x_b, c] = D[c, x_b]
        labels.append((xb, bond))
        raw.append(ng + n + 2 * g + 1)
        cur[a], cur[b] = xb, xa
    for q in range(n):
        if q in open_qubits:
            continue
        v = np.zeros(2, dtype=np.complex128)
        v[int(bits[q])] = 1.0
        tensors.append(v)
        labels.append((cur[q],))
        raw.append(-(q + 1))
    net = HyperNetwork(tensors, labels, [cur[q] for q in open_qubits], raw)
    net.producer = producer
    net.final = list(cur)
    return net


def fix_indices(net, fixed):
    """Slice: give each index in ``fixed`` (name -> 0/1) its value in every
    tensor that holds it."""
    tensors, labels = [], []
    for T, ls in zip(net.tensors, net.labels):
        idx = tuple(int(fixed[l]) if l in fixed else slice(None) for l in ls)
        tensors.append(T[idx] if ls else T)
        labels.append(tuple(l for l in ls if l not in fixed))
    out = HyperNetwork(tensors, labels, net.open_labels, net.raw)
    out.producer, out.final = getattr(net, "producer", None), getattr(net, "final", None)
    return out


def contract_pair(A, la, B, lb, keep):
    """Product of A and B summed over the shared indices that are not in
    ``keep`` (``keep``: indices some other tensor or the output still needs).
    Shared indices in ``keep`` are batch indices:
        C[b, m, n] = sum_k A[b, m, k] B[b, k, n]
    (numpy.matmul over the batch); result indices: batch, A's free, B's free."""
    la, lb = tuple(la), tuple(lb)
    shared = [l for l in la if l in lb]
    batch = [l for l in shared if l in keep]
    summed = [l for l in shared if l not in keep]
    free_a = [l for l in la if l not in lb]
    free_b = [l for l in lb if l not in la]
    a = np.transpose(A, [la.index(l) for l in batch + free_a + summed]) if la else A
    b = np.transpose(B, [lb.index(l) for l in batch + summed + free_b]) if lb else B
    nb, nm, nk, nn = 2 ** len(batch), 2 ** len(free_a), 2 ** len(summed), 2 ** len(free_b)
    c = np.matmul(a.reshape(nb, nm, nk), b.reshape(nb, nk, nn))
    lc = tuple(batch + free_a + free_b)
    return c.reshape((2,) * len(lc)) if lc else c.reshape(()), lc


def contract_tree(tensors, labels, open_labels, pairs):
    """Contract in the SSA order ``pairs`` (inputs 0..L-1, pair i -> L + i);
    a pair sums an index when no tensor outside the pair and no open output
    holds it, and keeps it otherwise."""
    store = {i: (t, tuple(l)) for i, (t, l) in enumerate(zip(tensors, labels))}
    holders = defaultdict(int)
    for l in labels:
        for x in l:
            holders[x] += 1
    opened = set(open_labels)
    nid = len(tensors)
    for i, j in pairs:
        (A, la), (B, lb) = store.pop(i), store.pop(j)
        for x in set(la) | set(lb):
            holders[x] -= (x in la) + (x in lb)
        keep = {x for x in set(la) | set(lb) if holders[x] > 0 or x in opened}
        C, lc = contract_pair(A, la, B, lb, keep)
        for x in lc:
            holders[x] += 1
        store[nid] = (C, lc)
        nid += 1
    assert len(store) == 1, "tree does not join every tensor"
    return next(iter(store.values()))


def greedy_pairs(labels):
    """An order of this module's own: repeatedly join the two tensors that
    share an index and give the smallest product (ties: smallest ids);
    disconnected pieces last.  Sizes are estimated from index counts."""
    active = {i: frozenset(l) for i, l in enumerate(labels)}
    pairs, nid = [], len(labels)
    while len(active) > 1:
        best = None
        ids = sorted(active)
        for x in range(len(ids)):
            for y in range(x + 1, len(ids)):
                i, j = ids[x], ids[y]
                if active[i] & active[j]:
                    key = (len(active[i] | active[j]), i, j)
                    if best is None or key < best:
                        best = key
        if best is None:
            i, j = ids[0], ids[1]
        else:
            _, i, j = best
        active[nid] = active.pop(i) | active.pop(j)
        pairs.append((i, j))
        nid += 1
    return pairs


def contract(net, pairs=None):
    """Amplitude vector (bit t of the index = open qubit t)."""
    if pairs is None:
        pairs = greedy_pairs(net.labels)
    if len(net.tensors) == 1:
        T, lt = net.tensors[0], net.labels[0]
    else:
        T, lt = contract_tree(net.tensors, net.labels, net.open_labels, pairs)
    return OTN.output_vector(T, lt, net.open_labels)


def amplitudes(gates, n, bit_rows, open_qubits=(), sliced=None, slice_ids=None):
    """complex128 (nb, 2^k) amplitudes of the decomposed network; with
    ``sliced`` (index names) the sum over ``slice_ids`` (default: all
    assignments; id s gives index j the value (s >> j) & 1)."""
    out = []
    for bits in bit_rows:
        net = circuit_network_split(gates, n, bits, open_qubits)
        if not sliced:
            out.append(contract(net))
            continue
        ids = range(1 << len(sliced)) if slice_ids is None else slice_ids
        acc = None
        for s in ids:
            v = contract(fix_indices(net, {l: (s >> j) & 1 for j, l in enumerate(sliced)}))
            acc = v if acc is None else acc + v
        out.append(acc)
    return np.array(out)


def contract_in_order(gates, n, bits, open_q, leaf_groups, pairs, fixed=None):
    """Replay a plan tree over the decomposed network: ``leaf_groups`` lists
    raw ids per leaf (as above; a closed qubit's projector joins the group
    holding the tensor that produced its final wire), ``pairs`` joins the
    groups.  The tree is only a schedule: the tensors and the arithmetic are
    this module's."""
    net = circuit_network_split(gates, n, bits, open_q)
    final_producer = {q: net.producer[net.final[q]] for q in range(n) if q not in open_q}
    if fixed:
        net = fix_indices(net, fixed)
    by_raw = defaultdict(list)
    for i, r in enumerate(net.raw):
        by_raw[r].append(i)
    members = []
    for raws in leaf_groups:
        m = [i for r in raws for i in by_raw[r]]
        m += [i for q, pr in final_producer.items() if pr in raws for i in by_raw[-(q + 1)]]
        members.append(m)
    # indices held outside each group, or open, stay in the group's tensor
    count = defaultdict(int)
    for ls in net.labels:
        for x in ls:
            count[x] += 1
    tens, labs = [], []
    for m in members:
        sub_t = [net.tensors[i] for i in m]
        sub_l = [net.labels[i] for i in m]
        inside = defaultdict(int)
        for ls in sub_l:
            for x in ls:
                inside[x] += 1
        outside = [x for x in inside if count[x] > inside[x]]
        if len(m) == 1:
            t, l = sub_t[0], sub_l[0]
        else:
            t, l = contract_tree(sub_t, sub_l, list(net.open_labels) + outside, greedy_pairs(sub_l))
        tens.append(t)
        labs.append(l)
    if pairs:
        t, l = contract_tree(tens, labs, net.open_labels, pairs)
    else:
        t, l = tens[0], labs[0]
    return OTN.output_vector(t, l, net.open_labels)
