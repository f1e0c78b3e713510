"""One process per GPU, each building and sampling its own independent table.

A single alias table does not shard without an exchange step, so the
multi-GPU form of the hot path is replicas: rank r works on its own weights
(seed + r), there is no collective on the data path, and the only
communication is a barrier around the timed region and a max over ranks of
the measured times (weak scaling: every rank does the same work, the job's
throughput is the units of all ranks over the slowest rank's time).

The process group is the caller's (NCCL on GPUs, gloo on CPUs); these
helpers only read the launcher's environment and do the reductions.
"""
from __future__ import annotations

import os


def env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s weights: independent tables per rank."""
    return base + rank


def max_over_ranks(values, group_dist=None, device=None) -> list[float]:
    """Element-wise maximum of `values` over all ranks (the slowest rank
    decides a weak-scaling time); identity without a process group."""
    vals = [float(v) for v in values]
    if group_dist is None:
        return vals
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    group_dist.all_reduce(t, op=group_dist.ReduceOp.MAX)
    return t.tolist()


def job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: the units of all ranks over the slowest time."""
    return world * units_per_rank / (ms_max / 1e3)
