"""Sharding one amplitude request over several GPUs (one process per GPU).

Slices are independent sub-tasks (Sec. "A Customized Parallelization
Scheme"); the only exchange is the final reduction of the amplitude vector
(Sec. "Scaling").  Rank r of a world of w contracts a contiguous range of slice
ids on its own GPU; the partial sums, nb * 2^k complex128 values per rank, are
all-gathered through the host (a gloo process group: at most a few hundred
KiB, so no GPU collective, peer access or NCCL is involved) and added in rank
order on every rank, so the result depends only on the world size, not on
the order in which the collective combines them.  With one rank it is the
plain single-GPU sum.
"""
import numpy as np


def slice_range(rank, world, num_slices):
    """[begin, end) of the slice ids of `rank` in a world of `world` ranks:
    contiguous ranges in rank order, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or num_slices < 0:
        raise ValueError(f"bad shard {rank}/{world} of {num_slices} slices")
    q, r = divmod(num_slices, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def reduce_in_rank_order(partial, group=None):
    """Sum over the ranks of `group` (a gloo process group) of each rank's
    complex128 partial amplitudes, added in rank order (identical on every
    rank)."""
    import torch
    import torch.distributed as dist
    if dist.get_backend(group) != "gloo":
        raise ValueError("the amplitude reduction runs on the host: pass a gloo process group")
    part = np.ascontiguousarray(partial, dtype=np.complex128)
    t = torch.from_numpy(part.view(np.float64).copy())
    bufs = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(bufs, t, group=group)
    acc = np.zeros_like(part)
    for b in bufs:
        acc += b.cpu().numpy().view(np.complex128).reshape(part.shape)
    return acc


def contract_sharded(plan, bitstrings, group=None, **kw):
    """This rank's slice range of `plan` (on the current GPU), then the
    rank-ordered reduction; keyword arguments go to contract_amplitudes."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    begin, end = slice_range(rank, world, plan.info()["num_slices"])
    part = plan.contract_amplitudes(bitstrings, slice_begin=begin, slice_count=end - begin, **kw)
    return reduce_in_rank_order(part, group)
