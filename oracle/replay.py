"""Oracle contraction in an externally given order.

The exact value of a tensor-network contraction does not depend on the order
in which pairs are contracted (pinned by the order-independence test), so for
networks where the oracle's own greedy order is too wide to run, the oracle
may follow a given tree.  The tensors, their index names, the fixing of sliced
indices and all arithmetic remain the oracle's own (``oracle.tn``); the tree
is only a schedule: a list of leaf groups (each a list of raw tensors) and SSA
pairs joining the groups.

Raw tensor ids: ``g < num_gates`` is gate g; ``num_gates + q`` is the |0>
input of qubit q.  The projector <x_q| of a closed qubit joins the group that
holds the last gate on q (or its input when q has no gate).
"""
from . import tn as OTN


def contract_in_order(gates, n, bits, open_q, leaf_groups, pairs, fixed=None):
    onet = OTN.circuit_network(gates, n, bits, open_q)
    if fixed:
        onet = OTN.fix_indices(onet, fixed)
    ng = len(gates)
    last_raw = {q: ng + q for q in range(n)}
    for gi, g in enumerate(gates):
        for q in g.qubits:
            last_raw[q] = gi
    closed = [q for q in range(n) if q not in open_q]
    proj_index = {q: n + ng + i for i, q in enumerate(closed)}
    tens, labs = [], []
    for raws in leaf_groups:
        grp = [r + n if r < ng else r - ng for r in raws]
        grp += [proj_index[q] for q in closed if last_raw[q] in raws]
        sub_t = [onet.tensors[i] for i in grp]
        sub_l = [onet.labels[i] for i in grp]
        if len(grp) > 1:
            t, l = OTN.contract_tree(sub_t, sub_l, OTN.greedy_order(sub_l))
        else:
            t, l = sub_t[0], sub_l[0]
        tens.append(t)
        labs.append(l)
    if pairs:
        t, l = OTN.contract_tree(tens, labs, pairs)
    else:
        t, l = tens[0], labs[0]
    return OTN.output_vector(t, l, onet.open_labels)


def work_cmac(gates, n, bits, open_q, leaf_groups, pairs, fixed=None):
    """Complex multiply-adds of the pairwise steps between groups (2^|A u B| each)."""
    onet = OTN.circuit_network(gates, n, bits, open_q)
    if fixed:
        onet = OTN.fix_indices(onet, fixed)
    ng = len(gates)
    last_raw = {q: ng + q for q in range(n)}
    for gi, g in enumerate(gates):
        for q in g.qubits:
            last_raw[q] = gi
    closed = [q for q in range(n) if q not in open_q]
    proj_index = {q: n + ng + i for i, q in enumerate(closed)}
    sets = []
    for raws in leaf_groups:
        grp = [r + n if r < ng else r - ng for r in raws]
        grp += [proj_index[q] for q in closed if last_raw[q] in raws]
        s = set()
        for i in grp:
            s ^= set(onet.labels[i])
        sets.append(frozenset(s))
    total = 0.0
    for i, j in pairs:
        a, b = sets[i], sets[j]
        total += 2.0 ** len(a | b)
        sets.append(a ^ b)
    return total
