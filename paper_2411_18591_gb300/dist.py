"""Data parallelism over fields: one process per GPU, each with its own shard of the batch.

The fields of a batch are independent, so forward and backward propagations need no
exchange between ranks. A parameter shared by every field (the pupil phase of the 4f
system, a diffractive mask) gets one gradient per rank from that rank's fields; the
gradient of the mean loss over the global batch is the mean of those (equal shards),
which is the single all-reduce of a step.
"""
from __future__ import annotations

import torch


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous, balanced share of ``n_items`` for ``rank`` of ``world`` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def average_gradient(grad: torch.Tensor, group=None) -> torch.Tensor:
    """In place: the mean over ranks of a shared parameter's gradient (one all-reduce)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if world > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
        grad.div_(world)
    return grad
