"""Sharding a uniform batch over ranks.

The pairs of Eq. (1) are independent (Section 2), so a batch splits into
contiguous ranges of pairs with no exchange between ranks: rank r computes
pairs [start, start + count) by calling the library with its operands offset
by start*ld2 elements.  The only collective a multi-rank run needs is the
timing reduction (the slowest rank's elapsed time).
"""
from __future__ import annotations


def shard_range(batch: int, rank: int, world: int) -> tuple[int, int]:
    """(start, count) of rank's share: the first batch % world ranks get one
    pair more than the rest."""
    if world < 1 or not 0 <= rank < world or batch < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(batch, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def shard_offsets(batch: int, rank: int, world: int, lda2: int, ldb2: int, ldc2: int,
                  elem_bytes: int):
    """Byte offsets of rank's A, B, C sub-batches and its pair count (A or B
    shared by all pairs when its ld2 is 0)."""
    start, count = shard_range(batch, rank, world)
    return (start * lda2 * elem_bytes, start * ldb2 * elem_bytes, start * ldc2 * elem_bytes,
            count)


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks of the default process group (the
    timed region ends when the slowest rank does); the value itself when no
    group is initialised."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
