"""Multi-process helpers (one process per GPU).

The MatExPre path shards by independent units: the medium is replicated on
every rank and the sources (right-hand sides) are split among the ranks, each
of which solves its share with the batched solver on its own GPU.  Nothing is
exchanged on the data path; the only collectives are the final gather of the
per-source results and the combination of the timings (the job's time is the
slowest rank's, its work the sum).
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


def _distributed():
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def reduce_job(seconds: float, units: float, device=None):
    """(max over ranks of seconds, sum over ranks of units); identity when not
    distributed.  Uses the default process group (gloo on CPU, nccl on GPU)."""
    import torch
    import torch.distributed as dist
    if not _distributed():
        return float(seconds), float(units)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def gather_by_index(local: dict, total: int):
    """Merge {unit index: result} from every rank into a list ordered by unit
    index (one all_gather of host objects); identity when not distributed.
    Raises if some unit has no result or two ranks report the same unit."""
    import torch.distributed as dist
    parts = [local]
    if _distributed():
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, local)
    out = [None] * total
    seen = set()
    for part in parts:
        for k, v in part.items():
            if k in seen or not 0 <= k < total:
                raise RuntimeError(f"unit {k} reported twice or out of range")
            seen.add(k)
            out[k] = v
    if len(seen) != total:
        raise RuntimeError(f"units without a result: {sorted(set(range(total)) - seen)}")
    return out


def solve_sharded(sources, solve_share, rank=None, world=None):
    """Solve many sources split across the ranks.

    sources     the job's right-hand sides, in a fixed order every rank agrees on
    solve_share callable(list of (index, source)) -> list of per-source results,
                run by each rank on its own share (on the GPU: the batched C-ABI
                solver on the rank's device, the medium replicated per rank)
    Returns every source's result, in source order, on every rank.
    """
    r0, w0, _ = env()
    rank = r0 if rank is None else rank
    world = w0 if world is None else world
    mine = shard(range(len(sources)), rank, world)
    results = solve_share([(i, sources[i]) for i in mine]) if mine else []
    if len(results) != len(mine):
        raise RuntimeError("solve_share returned a result count different from its share")
    return gather_by_index(dict(zip(mine, results)), len(sources))


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
