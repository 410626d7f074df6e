"""The multi-rank path of the benchmark on CPU: two gloo ranks shard cells with
no overlap and no gap, and the report reduces time by max and pairs by sum."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2206_02937_gb300.dist import reduce_timing, shard_cells


def test_shard_cells_cover_exactly():
    for n, world in ((10, 3), (262144, 8), (5, 8), (1, 1)):
        ranges = [shard_cells(n, r, world) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        for (a, b), (c, d) in zip(ranges, ranges[1:]):
            assert b == c and a <= b
        sizes = [b - a for a, b in ranges]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_cells(10, 3, 3)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = shard_cells(1000, rank, world)
        t, p = reduce_timing(10.0 + rank, float(hi - lo))
        q.put((rank, t, p))
    finally:
        dist.destroy_process_group()


def test_gloo_world2_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, p in out:
        assert t == 11.0 and p == 1000.0
    _ = torch
