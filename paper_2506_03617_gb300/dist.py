"""Multi-process helpers for weak-scaling runs (one process per GPU).

The MatExPre path shards by independent units (sources, media): every rank
solves its own share and nothing is exchanged on the data path.  Only the
timing is combined: the job's time is the slowest rank's, its work the sum.
"""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items, rank, world):
    """The units this rank owns: round-robin, every unit exactly once."""
    return list(items)[rank::world]


def reduce_job(seconds: float, units: float, device=None):
    """(max over ranks of seconds, sum over ranks of units); identity when not
    distributed.  Uses the default process group (gloo on CPU, nccl on GPU)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds), float(units)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
