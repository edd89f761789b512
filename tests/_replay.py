"""Test helper: oracle contraction of a library plan's tree (see oracle.replay)."""
from oracle.replay import contract_in_order


def replay(plan, gates, n, bits, open_q, fixed=None):
    leaves, pairs = plan.tree(len(gates), n)
    return contract_in_order(gates, n, bits, open_q, leaves, pairs, fixed)
