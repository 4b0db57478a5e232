"""Sharding a uniform or variable-size batch over ranks.

The pairs of Eq. (1) are independent (Section 2), so a batch splits into
contiguous ranges of pairs with no exchange between ranks: rank r computes
pairs [start, start + count) by calling the library with its operands offset
by start*ld2 elements.  A variable-size batch splits into contiguous runs of
its problems with near-equal estimated cost; each rank plans and runs its
own run on the same arenas.  The only collective a multi-rank run needs is
the timing reduction (the slowest rank's elapsed time).
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


def problem_costs(desc, elem_bytes: int):
    """Estimated cost of each problem of a variable-size batch (rows
    (m, n, k, flags, offA, offB, offC, 0), flags bit 4 = beta zero): its
    algorithmic bytes s*(mk + kn + mn*(1 + [beta != 0])), the quantity the
    memory-bound kernels move.  Any other per-problem estimate (for example
    the cost model's predicted times) can be passed to ``shard_problems``
    instead."""
    import numpy as np
    d = np.asarray(desc, dtype=np.int64)
    m, n, k = d[:, 0], d[:, 1], d[:, 2]
    bz = (d[:, 3] >> 4) & 1
    return elem_bytes * (m * k + k * n + m * n * (2 - bz))


def shard_problems(costs, world: int):
    """Boundaries b[0] = 0 <= ... <= b[world] = len(costs): rank r takes the
    contiguous problems [b[r], b[r + 1]), cut where the running cost reaches
    r / world of the total, so neighbouring problems of the arena stay on one
    rank and every rank's cost is within the largest single cost of an equal
    share."""
    import numpy as np
    if world < 1:
        raise ValueError("bad shard request")
    c = np.asarray(costs, dtype=np.float64)
    if c.ndim != 1 or np.any(c < 0):
        raise ValueError("costs must be a non-negative vector")
    prefix = np.concatenate([[0.0], np.cumsum(c)])
    total = prefix[-1]
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(prefix, total * r / world, side="left")))
    cuts.append(len(c))
    return np.maximum.accumulate(np.asarray(cuts, dtype=np.int64))
