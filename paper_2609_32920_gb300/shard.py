"""Path sharding across ranks (one process per GPU).

Light paths are independent, so N ranks trace disjoint ranges of the global path index
space with the estimator normalised by the total count; no collective is needed on the data
path (summing the ranks' images or gradients, if a caller wants the whole-job result, gives
exactly the single-process result).  The only collective the benchmark uses is the
max-over-ranks of its timings.
"""
from __future__ import annotations


def path_shard(rank: int, world: int, paths_per_rank: int):
    """(path_offset, n_paths, n_norm) for this rank: weak scaling, each rank its own
    contiguous range of `paths_per_rank` Philox counters."""
    if world < 1 or not 0 <= rank < world or paths_per_rank < 0:
        raise ValueError("bad shard request")
    return rank * paths_per_rank, paths_per_rank, paths_per_rank * world


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a scalar over all ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
