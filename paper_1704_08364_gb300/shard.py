"""Slice sharding across ranks (one process per GPU).

Slices are independent (each slice x(u1, u2) of the volume is reconstructed
from its own sinogram, Sec. 1), so the forward path shards by contiguous
slice ranges with no collective; ranges hold whole slice pairs (the kernels
transform two slices per complex line).  The only exchange of the
differentiable path is the sum of the filter-tap gradient over ranks.
"""
from __future__ import annotations


def slice_range(rank: int, world: int, slices: int) -> tuple[int, int]:
    """[start, stop) of this rank's slices: contiguous, whole pairs, sizes
    differing by at most one pair (the last range may end on an odd slice)."""
    if world <= 0 or not 0 <= rank < world or slices < 0:
        raise ValueError("bad rank/world/slices")
    pairs = (slices + 1) // 2
    base, extra = divmod(pairs, world)
    p0 = rank * base + min(rank, extra)
    p1 = p0 + base + (1 if rank < extra else 0)
    return min(2 * p0, slices), min(2 * p1, slices)


def allreduce_filter_grad(grad, group=None):
    """Sum the filter-tap gradient over the ranks of `group` (in place)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad
