"""Sharding of a particle stack across ranks (one process per GPU).

Alignment needs no communication: every image is independent given the
references.  The class average has one exchange step: each rank adds its
shard's compensated class sums and counts (``mra_class_sums``), the three
arrays are summed over ranks, and every rank finalises locally
(``mra_average_finalize``).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_range(n: int, world: int, rank: int):
    """Contiguous [begin, end) slice of n images for `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def allreduce_class_sums(sums: torch.Tensor, comp: torch.Tensor, counts: torch.Tensor, group=None) -> None:
    """Sum the per-class (sum, correction, count) arrays over all ranks, in place."""
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return
    for t in (sums, comp, counts):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
