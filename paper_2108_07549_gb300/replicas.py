"""Replica bookkeeping for a run on several GPUs of one node.

The PDR sweep does not shard: each rank solves its own replica of the
instance on its own GPU, with no data exchanged between ranks.  The host only
needs two reductions over the ranks: the slowest rank's time, and the
whole-job throughput, which is the sum of the ranks' updates over that time.
"""

from __future__ import annotations


def slowest(seconds: float, world: int, device="cpu") -> float:
    """The largest of `seconds` over all ranks (itself on a single rank).

    Every rank must call it (it is an all-reduce); `device` is where the
    process group's backend reduces (a CUDA device for NCCL, the CPU for gloo).
    """
    if world <= 1:
        return float(seconds)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(updates_per_rank: float, slowest_seconds: float, world: int) -> float:
    """Whole-job updates per second: every rank's updates over the slowest rank's time."""
    return max(world, 1) * float(updates_per_rank) / float(slowest_seconds)
