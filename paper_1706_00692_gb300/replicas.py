"""Multi-GPU runs of the solver as independent replicas: one process per GPU
(launched by torchrun), each solving its own copy of the problem. The solve
has no data-path exchange, so the only collective is the timing reduction:
the job's time is the slowest rank's, and its throughput counts the units
(converged eigenpairs) of every rank."""
from __future__ import annotations

import os


def dist_env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment; (0, 1, 0)
    when not launched by torchrun."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not (0 <= rank < world) or local < 0:
        raise ValueError(f"bad rank environment: RANK={rank} WORLD_SIZE={world} LOCAL_RANK={local}")
    return rank, world, local


def job_throughput(local_units: float, local_seconds: float, device=None) -> tuple[float, float, float]:
    """Whole-job (units, seconds, units/s) of replicated runs: units summed over
    ranks, time = the slowest rank's. Every rank must call it (it holds the
    ranks together with a barrier first). Single-process runs return the local
    values. device: where the reduction tensors live (a CUDA device for NCCL,
    None for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_units), float(local_seconds), float(local_units) / float(local_seconds)
    dist.barrier()
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    units, secs = float(u.item()), float(t.item())
    return units, secs, units / secs
