"""Multi-process helpers of the benchmark (one process per GPU).

The Compton step is cell-local: pairing and collisions never cross a cell, so
ranks own disjoint sets of cells and exchange nothing inside a step.  The only
collective work is the reduction of the timing (max over ranks) and of the
processed-pair counts (sum) for the report.  These helpers are backend
agnostic (NCCL on GPUs, gloo on CPUs in the tests).
"""
from __future__ import annotations


def shard_cells(n_cells: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous cell range [lo, hi) of `rank` out of `world`: slabs of equal
    size, the first n_cells % world ranks one cell larger."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    base, extra = divmod(n_cells, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def reduce_timing(elapsed_ms: float, pairs: float, device=None) -> tuple[float, float]:
    """(max elapsed over ranks, sum of pairs over ranks); identity without a
    process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(elapsed_ms), float(pairs)
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    p = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())
