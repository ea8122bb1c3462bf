"""Host side of a run on several GPUs of one node, one process per GPU.

Every parameter instance of Eq. (1) is an independent problem (Algorithm 4 runs
per mu), so the ranks split the instances and exchange nothing on the data
path: each rank solves its own batch on its own GPU (weak scaling).  What the
ranks share is host bookkeeping only: which rows of the parameter set a rank
takes, the step time as the maximum over ranks, and the whole-job rate.
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass(frozen=True)
class RankInfo:
    rank: int
    world: int
    local: int


def rank_info(env=None) -> RankInfo:
    """RANK / WORLD_SIZE / LOCAL_RANK as set by torch.distributed.run (defaults: one process)."""
    env = os.environ if env is None else env
    info = RankInfo(int(env.get("RANK", "0")), int(env.get("WORLD_SIZE", "1")), int(env.get("LOCAL_RANK", "0")))
    if info.world < 1 or not 0 <= info.rank < info.world or info.local < 0:
        raise ValueError(f"inconsistent rank environment: {info}")
    return info


def shard(rows, per_rank: int, rank: int, world: int):
    """The contiguous block of `per_rank` rows that `rank` solves; `rows` holds the
    whole job's instances (per_rank * world of them), so the blocks of all ranks
    are disjoint and cover it."""
    if per_rank < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad shard request: per_rank={per_rank} rank={rank} world={world}")
    if len(rows) != per_rank * world:
        raise ValueError(f"{len(rows)} rows for {world} ranks of {per_rank}")
    return rows[rank * per_rank:(rank + 1) * per_rank]


def max_over_ranks(x: float, device=None) -> float:
    """max of x over the ranks of the initialised process group (x itself without one).
    `device` is where the one-element tensor lives: the rank's GPU under NCCL, the
    CPU under gloo."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job throughput in units/s: the units all ranks processed in one step
    divided by the slowest rank's step time."""
    if ms_per_step <= 0:
        raise ValueError("step time must be positive")
    return units_per_rank * world / (ms_per_step / 1e3)
