"""Oracle contraction of the library's plan tree on the oracle's own network.

The order of a contraction does not change its exact value (pinned by
test_tn_order_independence), so for networks where the oracle's own greedy
order is too wide, the oracle may follow the planner's tree: the tensors,
their index names and the arithmetic are still the oracle's own."""
from oracle import circuit as OC
from oracle import tn as OTN


def replay(plan, gates, n, bits, open_q, fixed=None):
    """Oracle value of the plan's network for one bitstring, with the wire
    segments in `fixed` ({(q, t): value}) fixed (a slice)."""
    onet = OTN.circuit_network(gates, n, bits, open_q)
    if fixed:
        onet = OTN.fix_indices(onet, fixed)
    ng = len(gates)
    leaves, pairs = plan.tree(ng, n)
    last_raw = {q: ng + q for q in range(n)}
    for gi, g in enumerate(gates):
        for q in g.qubits:
            last_raw[q] = gi
    closed = [q for q in range(n) if q not in open_q]
    proj_index = {q: n + ng + i for i, q in enumerate(closed)}
    tens, labs = [], []
    for raws in leaves:
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
