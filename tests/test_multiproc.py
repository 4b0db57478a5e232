"""Multi-rank host logic on CPU with the gloo backend (world size 2): the
sharded batch reproduces the unsharded result bit for bit, and the timing
reduction takes the slowest rank."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1304_7053_gb300 import shard


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_ranges_cover_batch_exactly():
    for N in (0, 1, 7, 1000, 100_003):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_range(N, r, world) for r in range(world)]
            assert sum(c for _, c in spans) == N
            pos = 0
            for s, c in spans:
                assert s == pos
                pos += c
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


def _worker(rank, world, port, q):
    import oracle
    from paper_1304_7053_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, N = 5, 1001
        b = inputs.UniformBatch("d", "T", "N", m, m, m, N, seed=3)
        oa, ob, oc, cnt = shard.shard_offsets(N, rank, world, b.lda2, b.ldb2, b.ldc2, 8)
        A = b.A[oa // 8:]
        B = b.B[ob // 8:]
        C = b.C[oc // 8:oc // 8 + cnt * b.ldc2]
        mine = oracle.gemm_uniform("d", "T", "N", m, m, m, 1.5, A, b.lda, b.lda2, B, b.ldb, b.ldb2,
                                   -0.5, C, b.ldc, b.ldc2, cnt)
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        elapsed = shard.max_over_ranks(10.0 + rank)
        if rank == 0:
            full = oracle.gemm_uniform("d", "T", "N", m, m, m, 1.5, b.A, b.lda, b.lda2, b.B, b.ldb,
                                       b.ldb2, -0.5, b.C, b.ldc, b.ldc2, N)
            q.put((bool(np.array_equal(np.concatenate(parts), full)), elapsed))
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_match_unsharded_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    same, elapsed = q.get(timeout=10)
    assert same
    assert elapsed == 11.0


def test_problem_shards_balance_cost():
    """Contiguous runs of a variable-size batch: they cover every problem once
    and each rank's estimated cost is within the largest single problem's
    cost of an equal share (the cut is placed at a prefix-sum crossing)."""
    from paper_1304_7053_gb300 import inputs
    desc, _, _, _ = inputs.vbatch_problems(5000, seed=4)
    costs = shard.problem_costs(desc, 4)
    m = desc[:, 0]
    bz = (desc[:, 3] >> 4) & 1
    assert np.array_equal(costs, 4 * m * m * (4 - bz))
    for world in (1, 2, 3, 7):
        b = shard.shard_problems(costs, world)
        assert b[0] == 0 and b[-1] == len(costs) and np.all(np.diff(b) >= 0)
        share = costs.sum() / world
        for r in range(world):
            assert abs(costs[b[r]:b[r + 1]].sum() - share) <= costs.max()
    assert list(shard.shard_problems([], 3)) == [0, 0, 0, 0]
    with pytest.raises(ValueError):
        shard.shard_problems([1.0, -1.0], 2)


def _vworker(rank, world, port, q):
    import oracle
    from paper_1304_7053_gb300 import inputs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        desc, la, lb, lc = inputs.vbatch_problems(3000, seed=5)
        A = inputs.draw("s", la, 11, int_valued=True)
        B = inputs.draw("s", lb, 12, int_valued=True)
        C = inputs.draw("s", lc, 13, int_valued=True)
        b = shard.shard_problems(shard.problem_costs(desc, 4), world)
        mine = desc[b[rank]:b[rank + 1]]
        out = oracle.gemm_vbatch("s", mine, 1.5, A, B, -0.5, C)
        spans = [(int(d[6]), out[d[6]:d[6] + d[0] * d[1]].copy()) for d in mine]
        parts = [None] * world
        dist.all_gather_object(parts, spans)
        if rank == 0:
            full = oracle.gemm_vbatch("s", desc, 1.5, A, B, -0.5, C)
            got = C.astype(np.float64)
            for p in parts:
                for off, v in p:
                    got[off:off + v.size] = v
            q.put(bool(np.array_equal(got, full)))
    finally:
        dist.destroy_process_group()


def test_two_rank_problem_shards_match_unsharded_gloo():
    """A variable-size batch split by estimated cost over two gloo ranks:
    the ranks' results, put back in the arena, equal the unsharded oracle
    result bit for bit (small-integer inputs)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_vworker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=10)
