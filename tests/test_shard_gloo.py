"""Multi-rank sharding of one request, run as world-size-2 gloo process
groups on the CPU: each rank contracts its contiguous slice range (here with
the oracle standing in for the GPU contraction) and the partial sums are
reduced in rank order."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import tn_inputs as I
from oracle import circuit as OC
from oracle import statevector as SV
from oracle import tn as OTN
from paper_2110_14502_gb300.shard import contract_sharded, reduce_in_rank_order, slice_range

ROWS, COLS, DEPTH, SEED = 3, 4, 8, 3
OPEN = (9, 10, 11)


def _problem():
    gates = OC.random_circuit(ROWS, COLS, DEPTH, SEED)
    n = ROWS * COLS
    words = I.bitstrings(n, 2, SEED)
    nets = [OTN.circuit_network(gates, n, I.bits_of(w, n), OPEN) for w in words]
    # five internal bond labels to slice (any labels give an exact sliced sum)
    wires = sorted({l for ls in nets[0].labels for l in ls})[3:8]
    return gates, n, words, nets, wires


class OraclePlan:
    """Stand-in for a library plan: the oracle's sliced contraction."""

    def __init__(self, nets, wires):
        self.nets, self.wires = nets, wires

    def info(self):
        return {"num_slices": 1 << len(self.wires)}

    def contract_amplitudes(self, bitstrings, slice_begin=0, slice_count=-1):
        ids = range(slice_begin, slice_begin + slice_count)
        return np.array([OTN.contract_sliced(net, self.wires, ids) for net in self.nets])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        gates, n, words, nets, wires = _problem()
        got = contract_sharded(OraclePlan(nets, wires), words)
        # a second reduction of rank-dependent values: rank order, on every rank
        order = reduce_in_rank_order(np.full(3, 10.0 ** rank, dtype=np.complex128))
        out.put((rank, got, order))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2])
def test_sharded_sum_equals_the_single_process_sum(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gates, n, words, nets, wires = _problem()
    full = np.array([OTN.contract_sliced(net, wires) for net in nets])
    ref = SV.amplitudes(SV.simulate(gates, n), n, [I.bits_of(w, n) for w in words], OPEN)
    for rank, got, order in sorted(res, key=lambda x: x[0]):
        assert np.linalg.norm(got - full) <= 1e-12 * np.linalg.norm(full)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
        assert np.allclose(order, sum(10.0 ** r for r in range(world)))
    # every rank holds the same bits
    assert all(np.array_equal(res[0][1], r[1]) for r in res)


def test_slice_ranges_partition_the_slices():
    for ns in (0, 1, 5, 1024, 4097):
        for world in (1, 2, 3, 8):
            got = [slice_range(r, world, ns) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == ns
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [e - b for b, e in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slice_range(2, 2, 8)
