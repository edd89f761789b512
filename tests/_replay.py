"""Test helper: oracle contraction of a library plan's tree (see oracle.replay
and, for networks built with the split diagonal, oracle.hyper)."""
from oracle.replay import contract_in_order


def replay(plan, gates, n, bits, open_q, fixed=None, split=False):
    leaves, pairs = plan.tree(len(gates), n)
    if split:
        from oracle import hyper
        return hyper.contract_in_order(gates, n, bits, open_q, leaves, pairs, fixed)
    return contract_in_order(gates, n, bits, open_q, leaves, pairs, fixed)
