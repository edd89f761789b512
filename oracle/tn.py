"""Independent FP64 tensor-network contractor.

The circuit becomes a tensor network (Sec. "Existing Efforts on Simulation of
RQCs", tensor approach): a one-qubit gate is a rank-2 tensor, a two-qubit gate
a rank-4 tensor, the input |0> of each qubit a rank-1 tensor and the
projector <x_q| of each closed output qubit a rank-1 tensor; open output
qubits leave their last wire as a free index.  Contracting every shared index
gives <x|U|0...0> (or the 2^k open amplitudes as a rank-k tensor).

Every index has dimension 2 and is named by its wire segment ``(q, t)``:
qubit ``q`` after its ``t``-th gate (``t = 0`` is the input wire).  These
names are independent of any implementation, so a set of sliced indices can
be stated as a list of ``(q, t)`` pairs.

Slicing (Sec. "A PEPS-based Simulation Method with an Optimized Slicing
Strategy"): fixing S indices to each of their 2^S value assignments splits
the contraction into 2^S independent ones whose sum is the unsliced result.
Here assignment ``s`` gives sliced index ``j`` the value ``(s >> j) & 1``.

Pairwise contraction uses ``numpy.tensordot``; the order is this module's own
greedy choice (smallest growth ``|C| - |A| - |B|`` first), unless a tree is
given to replay.
"""
from collections import defaultdict

import numpy as np


class Network:
    def __init__(self, tensors, labels, open_labels):
        self.tensors = list(tensors)      # ndarrays of shape (2,)*rank, complex128
        self.labels = [tuple(l) for l in labels]
        self.open_labels = list(open_labels)  # bit t of the output index <-> open_labels[t]


def circuit_network(gates, n, bits=None, open_qubits=()):
    """Network of <x|U|0^n> for one bitstring ``bits`` (length n; the values
    of open qubits are ignored)."""
    open_qubits = list(open_qubits)
    seg = [0] * n
    tensors, labels = [], []
    for q in range(n):
        tensors.append(np.array([1.0, 0.0], dtype=np.complex128))
        labels.append(((q, 0),))
    for g in gates:
        if len(g.qubits) == 1:
            (q,) = g.qubits
            w_in = (q, seg[q])
            seg[q] += 1
            tensors.append(np.array(g.matrix, dtype=np.complex128))      # [out, in]
            labels.append(((q, seg[q]), w_in))
        else:
            a, b = g.qubits
            ia, ib = (a, seg[a]), (b, seg[b])
            seg[a] += 1
            seg[b] += 1
            U4 = np.array(g.matrix, dtype=np.complex128).reshape(2, 2, 2, 2)  # [a', b', a, b]
            tensors.append(U4)
            labels.append(((a, seg[a]), (b, seg[b]), ia, ib))
    for q in range(n):
        if q in open_qubits:
            continue
        v = np.zeros(2, dtype=np.complex128)
        v[int(bits[q])] = 1.0
        tensors.append(v)
        labels.append(((q, seg[q]),))
    open_labels = [(q, seg[q]) for q in open_qubits]
    return Network(tensors, labels, open_labels)


def contract_pair(A, la, B, lb):
    shared = [l for l in la if l in lb]
    ia = [la.index(l) for l in shared]
    ib = [lb.index(l) for l in shared]
    C = np.tensordot(A, B, axes=(ia, ib))
    lc = tuple(l for l in la if l not in shared) + tuple(l for l in lb if l not in shared)
    return C, lc


def greedy_order(label_lists):
    """Contraction tree as SSA pairs: tensor ids 0..L-1 are the inputs, the
    result of pair number i gets id L+i.  Each step contracts the connected
    pair with the smallest growth 2^|C| - 2^|A| - 2^|B| (ties: smallest ids);
    disconnected pieces are joined last, smallest first."""
    active = {i: frozenset(l) for i, l in enumerate(label_lists)}
    holders = defaultdict(set)
    for i, s in active.items():
        for l in s:
            holders[l].add(i)
    pairs = []
    nid = len(label_lists)
    while len(active) > 1:
        best = None
        for l, hs in holders.items():
            hs = sorted(hs)
            for x in range(len(hs)):
                for y in range(x + 1, len(hs)):
                    i, j = hs[x], hs[y]
                    out = active[i] ^ active[j]
                    key = (2.0 ** len(out) - 2.0 ** len(active[i]) - 2.0 ** len(active[j]), i, j)
                    if best is None or key < best:
                        best = key
        if best is None:
            ids = sorted(active, key=lambda i: (len(active[i]), i))
            i, j = ids[0], ids[1]
        else:
            _, i, j = best
        out = active[i] ^ active[j]
        for l in active[i] | active[j]:
            holders[l].discard(i)
            holders[l].discard(j)
            if not holders[l]:
                del holders[l]
        del active[i], active[j]
        active[nid] = out
        for l in out:
            holders[l].add(nid)
        pairs.append((i, j))
        nid += 1
    return pairs


def contract_tree(tensors, labels, pairs):
    """Contract inputs in the SSA order ``pairs``; returns (array, labels)."""
    store = {i: (t, tuple(l)) for i, (t, l) in enumerate(zip(tensors, labels))}
    nid = len(tensors)
    for i, j in pairs:
        (A, la), (B, lb) = store.pop(i), store.pop(j)
        store[nid] = contract_pair(A, la, B, lb)
        nid += 1
    assert len(store) == 1, "tree does not join every tensor"
    return next(iter(store.values()))


def output_vector(T, lt, open_labels):
    """Arrange the final tensor so that flat index j has bit t = open_labels[t]."""
    assert set(lt) == set(open_labels), (lt, open_labels)
    if not open_labels:
        return np.array([complex(T)], dtype=np.complex128)
    axes = [lt.index(l) for l in reversed(open_labels)]
    return np.ascontiguousarray(np.transpose(T, axes)).reshape(-1)


def fix_indices(net, assignment):
    """Network with each label in ``assignment`` fixed to its value (the
    sliced sub-network of one assignment)."""
    tensors, labels = [], []
    for T, l in zip(net.tensors, net.labels):
        idx = tuple(assignment[x] if x in assignment else slice(None) for x in l)
        tensors.append(np.asarray(T[idx]))
        labels.append(tuple(x for x in l if x not in assignment))
    return Network(tensors, labels, net.open_labels)


def contract(net, pairs=None):
    if pairs is None:
        pairs = greedy_order(net.labels)
    T, lt = contract_tree(net.tensors, net.labels, pairs)
    return output_vector(T, lt, net.open_labels)


def slice_assignment(sliced, s):
    return {lab: (s >> j) & 1 for j, lab in enumerate(sliced)}


def contract_slice(net, sliced, s, pairs=None):
    """Contribution of slice ``s``: sliced[j] fixed to bit j of s."""
    sub = fix_indices(net, slice_assignment(sliced, s))
    return contract(sub, pairs)


def contract_sliced(net, sliced, slice_ids=None):
    """Sum of the slice contributions over ``slice_ids`` (default: all 2^S),
    accumulated in slice-id order.  One greedy order serves every slice."""
    sliced = list(sliced)
    if slice_ids is None:
        slice_ids = range(1 << len(sliced))
    slice_ids = list(slice_ids)
    sub0 = fix_indices(net, slice_assignment(sliced, 0))
    pairs = greedy_order(sub0.labels)
    acc = None
    for s in slice_ids:
        v = contract_slice(net, sliced, s, pairs)
        acc = v if acc is None else acc + v
    return acc


def amplitudes(gates, n, bit_rows, open_qubits=(), sliced=None, slice_ids=None):
    """complex128 (nb, 2^k) amplitudes by tensor contraction."""
    out = []
    for bits in bit_rows:
        net = circuit_network(gates, n, bits, open_qubits)
        if sliced:
            out.append(contract_sliced(net, sliced, slice_ids))
        else:
            out.append(contract(net))
    return np.array(out)
