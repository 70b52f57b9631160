"""Query-parallel execution over several GPUs, one process per GPU.

Range queries are independent (Alg. 6 is a parallel for over queries), so the
path shards without any data-path collective: every rank holds a replica of
the index and answers its own queries.  The only cross-rank operations are a
barrier and the max of the step time, used for whole-job throughput.
"""
from __future__ import annotations


def shard_bounds(nq: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous share [lo, hi) of nq queries for `rank` (sizes differ by at most one)."""
    base, extra = divmod(nq, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def rank_query_seed(base_seed: int, rank: int) -> int:
    """Seed of the query batch a rank draws under weak scaling (rank 0 keeps the base batch)."""
    return base_seed + 1 + 7919 * rank


def reduce_max(value: float, device=None) -> float:
    """Max of a float over all ranks of the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, max_ms: float) -> float:
    """Units all ranks processed per second, timed by the slowest rank."""
    return units_per_rank * world / (max_ms / 1000.0)
