"""Process layout of a multi-GPU run.

One process per GPU.  The scenes of a batch are independent problems (each has
its own planes, views and supervision), so ranks shard scenes and exchange no
data on the splatting path: no collective runs between the kernels of a step.
The only cross-rank traffic is bookkeeping around the timed region, a barrier
before it and a maximum of the per-rank times after it, so that the job's time
is the slowest rank's.
"""
from __future__ import annotations

import torch


def scene_shard(n_scenes: int, rank: int, world: int) -> range:
    """Contiguous block of scene indices owned by `rank` (sizes differ by at
    most one; every scene is owned by exactly one rank)."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("rank %d outside world %d" % (rank, world))
    base, extra = divmod(max(n_scenes, 0), world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def rank_seeds(rank: int) -> dict:
    """Seeds of the scene a rank fits in the throughput run (weak scaling: each
    rank renders its own room of the same size)."""
    return {"scene": 1000 + rank, "init": 2000 + rank}


def _active() -> bool:
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def barrier() -> None:
    if _active():
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, device="cpu") -> float:
    """Maximum of a per-rank scalar over all ranks (identity on one process)."""
    if not _active():
        return float(x)
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device="cpu") -> float:
    """Sum of a per-rank scalar over all ranks (identity on one process)."""
    if not _active():
        return float(x)
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_all_ranks: float, max_seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time."""
    if max_seconds <= 0:
        raise ValueError("non-positive time")
    return units_all_ranks / max_seconds
