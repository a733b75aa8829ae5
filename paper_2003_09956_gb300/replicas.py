"""Multi-GPU benchmark runs as independent replicas (one process per GPU).

Every rank solves its own system.  The row-sharded form of one system
(the exchange of each worker's y, h and maxima every iteration) is in
shard.py; the benchmark's multi-GPU runs use replicas.  The only
cross-rank steps here are timing ones: a barrier before and after the
timed region and the maximum of the ranks' times, so `value` = units
processed by all ranks / slowest rank's time.  Works with any
torch.distributed backend (nccl on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import os


def rank_info() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def barrier(dist) -> None:
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float, device=None) -> float:
    """The largest value over all ranks (the identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world: int, units_per_rank: float, max_seconds: float) -> float:
    """Whole-job throughput: every rank processed units_per_rank in at most max_seconds."""
    return world * units_per_rank / max_seconds
