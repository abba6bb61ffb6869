"""Host-side logic of the multi-GPU split (one process per GPU).

The test pass partitions into independent matrices (problem 1.1 is solved
for every d on its own), so ranks take disjoint contiguous shards and need
no collective.  The training side has one exchange: the mode-1 Gram matrix
is a sum over the training matrices (Section 3.1, Eq. 3.2), so each rank
forms the partial Gram of its shard and the partials are summed with one
all-reduce before every rank extracts the same sketch.
"""
from __future__ import annotations

from typing import Tuple

import torch


def shard_range(count: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous [start, stop) of `count` items owned by `rank` of `world`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def allreduce_gram(G: torch.Tensor, group=None) -> torch.Tensor:
    """Sums the ranks' partial Gram matrices in place (float64)."""
    import torch.distributed as dist
    if G.dtype != torch.float64:
        raise ValueError("Gram partials are float64")
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(G, op=dist.ReduceOp.SUM, group=group)
    return G
