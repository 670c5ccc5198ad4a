"""Host-side logic of the multi-GPU form: independent replicas, no data-path collective.

The packet split shards without any exchange (Sec. IV.A: every node holds the
whole rule list and processes its own packets), so N GPUs run N replicas.
Each rank draws its own batch (weak scaling), times its own steps, and the
only collectives are a barrier around the timed region and a max over ranks
of the elapsed time, from which the whole-job rate is formed.
"""
from __future__ import annotations

import os


def world():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def packets_seed(base_seed: int, rank: int) -> int:
    """Seed of rank ``rank``'s packet batch: distinct per rank, rank 0 uses the base seed."""
    return int(base_seed) + 1000 * int(rank)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of ``value`` over all ranks (identity without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(packets_per_rank: int, steps: int, world_size: int, max_elapsed_ms: float) -> float:
    """Whole-job Mpackets/s: all ranks' packets over the slowest rank's elapsed time."""
    return world_size * packets_per_rank * steps / (max_elapsed_ms * 1e-3) / 1e6
