"""Multi-GPU layout of the sensor step: one process per GPU, envs sharded by
rank with no exchange on the data path.

Envs are independent, and every random draw is keyed by the global taxel id
(per taxel) or the global env id (per env), so a rank that simulates its own
block of envs with globally unique ids reproduces exactly what one process
holding all blocks would compute.  The only collective is the timing
reduction (max over ranks).
"""
from __future__ import annotations

import os


def rank_env():
    """(world size, rank, local rank) from the launcher's environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_ids(rank: int, n_envs: int, n_taxels: int):
    """(taxel_gid0, env_gid0) of rank `rank` when every rank holds n_envs envs
    with n_taxels taxels in all: rank r's ids follow rank r - 1's."""
    if rank < 0 or n_envs < 0 or n_taxels < 0:
        raise ValueError("rank, n_envs and n_taxels must be >= 0")
    return rank * n_taxels, rank * n_envs


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of `value` over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
