"""Whole-job timing of independent replicas (one process per GPU).

The pipeline does not shard: a diagram is one global reduction.  Under
torchrun each rank computes its own field, and the job's throughput is the
units all ranks processed divided by the slowest rank's time (weak scaling,
no collective on the data path: only these two reductions of the timing).
"""
from __future__ import annotations


def world():
    """(world size, rank) of the initialised process group, else (1, 0)."""
    try:
        import torch.distributed as dist
    except ImportError:  # pragma: no cover
        return 1, 0
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(), dist.get_rank()
    return 1, 0


def max_over_ranks(ms: float, device="cpu") -> float:
    """The largest per-step time over all ranks (every rank gets it)."""
    ws, _ = world()
    if ws == 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, max_ms: float) -> float:
    """Units per second of the whole job: every rank's units over the
    slowest rank's time."""
    ws, _ = world()
    return ws * float(units_per_rank) / (float(max_ms) * 1e-3)
