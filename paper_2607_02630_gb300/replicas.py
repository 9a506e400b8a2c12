"""Replica bookkeeping for runs on several GPUs.

The offload shards without any exchange step: requests are independent, so
every rank encrypts its own copy of the workload on its own GPU (weak
scaling, no collective on the data path).  The only collectives are the
barrier around the timed region and a MAX of the per-rank elapsed times, so
that the reported throughput is all ranks' bytes over the slowest rank.
"""
from __future__ import annotations

import os


def world_from_env(env=None) -> tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment."""
    env = os.environ if env is None else env
    return int(env.get("WORLD_SIZE", "1")), int(env.get("RANK", "0")), int(env.get("LOCAL_RANK", "0"))


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank's replica: independent requests per rank."""
    return base + 1000 * rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (the value itself without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gbs(bytes_per_rank: int, steps: int, world_size: int, max_elapsed_s: float) -> float:
    """Whole-job throughput: every rank's bytes over the slowest rank's time."""
    return world_size * bytes_per_rank * steps / max_elapsed_s / 1e9
