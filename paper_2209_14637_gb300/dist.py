"""Host-side logic of the multi-GPU split (one process per GPU).

The test pass partitions into independent matrices (problem 1.1 is solved
for every d on its own), so ranks take disjoint contiguous shards and need
no collective.  The training side has one exchange: the mode-1 Gram matrix
is a sum over the training matrices (Section 3.1, Eq. 3.2), so each rank
forms the partial Gram of its shard and the partials are summed with one
all-reduce before every rank extracts the same sketch.  The learned refiner
(Eq. 2.1) is data-parallel SGD: each rank takes an equal share of every
batch, and the gradients of the per-rank mean losses are averaged over the
ranks, which gives the gradient of the mean loss over the whole batch.
"""
from __future__ import annotations

from typing import Callable, Tuple

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


def allreduce_mean(t: torch.Tensor, group=None) -> torch.Tensor:
    """Averages a floating-point tensor over the ranks, in place."""
    import torch.distributed as dist
    if not t.is_floating_point():
        raise ValueError("only floating-point tensors are averaged")
    if dist.is_available() and dist.is_initialized():
        world = dist.get_world_size(group)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            t /= world
    return t


def data_parallel_sgd(grad_fn: Callable, S0: torch.Tensor, batch_of: Callable, steps: int,
                      lr: float, group=None) -> torch.Tensor:
    """Plain SGD on S = S0 + dS (dS starts at zero) with the gradient averaged
    over the ranks each step.

    grad_fn(S, batch) returns the gradient (shaped like S) of the mean loss
    over `batch`, this rank's share of the step's batch (`batch_of(step)`);
    the shares must have equal sizes on all ranks for the average to be the
    gradient of the whole batch's mean loss.  Every rank returns the same dS.
    """
    dS = torch.zeros_like(S0)
    for step in range(steps):
        g = grad_fn(S0 + dS, batch_of(step))
        allreduce_mean(g, group)
        dS -= lr * g
    return dS
