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


# ------------------------------------------------------------- slab decomposition
# One grid split into slabs of rows of its last axis (y in 2D, z in 3D), one per
# rank, as in the paper's distributed runs (Sec. 4).  Each rank keeps its owned
# rows plus `halo` rows of each neighbour.  A Taylor-Horner step on the extended
# slab is exact on every row at least one row away from the slab's outer edge;
# after K <= halo steps the owned rows are still exact, so the ranks exchange
# their edge rows every `halo` steps (and at every sub-step end, where y is
# taken from p).  The Krylov dot products need one sum over the ranks.


def slab_bounds(n_rows: int, world: int):
    """Owned rows [r0, r1) of every rank: a balanced split of n_rows."""
    base, extra = divmod(int(n_rows), int(world))
    out, r = [], 0
    for k in range(world):
        m = base + (1 if k < extra else 0)
        out.append((r, r + m))
        r += m
    return out


def slab_extended(bounds, rank: int, halo: int, n_rows: int):
    """Rows [e0, e1) a rank holds: its owned rows plus `halo` rows of each neighbour."""
    r0, r1 = bounds[rank]
    return max(0, r0 - halo), min(int(n_rows), r1 + halo)


class SlabExchange:
    """Exchange of `halo` edge rows between neighbouring slabs over
    torch.distributed point-to-point operations (gloo for CPU tensors, nccl for
    CUDA tensors), one slab per rank.  Vectors hold the extended slab, x
    fastest, `row_len` values per row; called with the list of this rank's
    vectors (one)."""

    def __init__(self, bounds, rank: int, halo: int, row_len: int, n_rows: int):
        self.bounds, self.rank, self.halo, self.row_len = bounds, int(rank), int(halo), int(row_len)
        self.world = len(bounds)
        for r0, r1 in bounds:
            if r1 - r0 < halo:
                raise ValueError("every slab must own at least `halo` rows")
        self.e0, self.e1 = slab_extended(bounds, rank, halo, n_rows)
        self.r0, self.r1 = bounds[rank]

    def _rows(self, v, a, b):
        """The rows [a, b) (global indices) of the extended-slab vector v."""
        return v[(a - self.e0) * self.row_len:(b - self.e0) * self.row_len]

    def __call__(self, vs):
        import torch.distributed as dist
        v = vs[0]
        reqs = []
        lo, hi = self.rank - 1, self.rank + 1
        if lo >= 0:
            reqs.append(dist.isend(self._rows(v, self.r0, self.r0 + self.halo).contiguous(), lo))
            reqs.append(dist.irecv(self._rows(v, self.e0, self.r0), lo))
        if hi < self.world:
            reqs.append(dist.isend(self._rows(v, self.r1 - self.halo, self.r1).contiguous(), hi))
            reqs.append(dist.irecv(self._rows(v, self.r1, self.e1), hi))
        for r in reqs:
            r.wait()


class LocalSlabExchange:
    """The same exchange for all slabs of a grid held by one process (the
    vectors of every slab, in slab order): halo rows are copied from the
    neighbouring slab's owned rows."""

    def __init__(self, bounds, halo: int, row_len: int, n_rows: int):
        self.bounds, self.halo, self.row_len = bounds, int(halo), int(row_len)
        for r0, r1 in bounds:
            if r1 - r0 < halo:
                raise ValueError("every slab must own at least `halo` rows")
        self.ext = [slab_extended(bounds, k, halo, n_rows) for k in range(len(bounds))]

    def _rows(self, k, v, a, b):
        e0 = self.ext[k][0]
        return v[(a - e0) * self.row_len:(b - e0) * self.row_len]

    def __call__(self, vs):
        for k in range(len(vs) - 1):
            r1 = self.bounds[k][1]                     # boundary between slab k and k + 1
            e1 = self.ext[k][1]
            e0n = self.ext[k + 1][0]
            self._rows(k, vs[k], r1, e1).copy_(self._rows(k + 1, vs[k + 1], r1, e1))
            self._rows(k + 1, vs[k + 1], e0n, r1).copy_(self._rows(k, vs[k], e0n, r1))


def slab_exp_action(steps, plan, t, p0s, bufs, exchange, halo):
    """exp(i t A_s) x on extended slabs by the sub-stepped Taylor-Horner
    recurrence (Def. psi; the plan (mu, S, m) of the whole grid):
      per sub-step, y = p at its start, then p <- y + i t / (S k) (A_s - mu) p for
      k = m .. 1, the last step of the last sub-step multiplied by e^{i t mu}.
    For every slab this process holds: steps[i](sigma, p, y, rho, out) computes
    out = rho (y + sigma (A_s - mu) p) on the extended slab (mxp_horner_step of a
    slab problem), p0s[i] holds x on the extended slab (halo rows are filled by
    the first exchange), bufs[i] two more vectors of the same size.
    exchange(list of vectors) refreshes the halo rows.  Returns, per slab, the
    vector that holds the result (its owned rows are exact)."""
    import cmath
    mu, S, m = plan
    rho_end = cmath.exp(1j * t * mu)
    ns = len(p0s)
    vecs = [[p0s[i], bufs[i][0], bufs[i][1]] for i in range(ns)]
    exchange([v[0] for v in vecs])
    iy = 0                                      # index of y (the sub-step start)
    for sub in range(S):
        cur, since = iy, 0
        for k in range(m, 0, -1):
            if since == halo:
                exchange([v[cur] for v in vecs])
                since = 0
            out = (iy + 1) % 3 if cur == iy else 3 - iy - cur
            rho = rho_end if (sub == S - 1 and k == 1) else 1.0
            for i in range(ns):
                steps[i](1j * t / (S * k), vecs[i][cur], vecs[i][iy], rho, vecs[i][out])
            cur = out
            since += 1
        if sub < S - 1:
            exchange([v[cur] for v in vecs])    # the next y needs exact halo rows
        iy = cur
    return [v[iy] for v in vecs]


def slab_dot(a, b, owned):
    """sum over the whole grid of conj(a) b for vectors split into slabs: the
    local sum over this rank's owned rows (`owned`, a slice of the extended
    slab) and one all_reduce (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    loc = torch.vdot(a[owned], b[owned])
    if not _distributed():
        return complex(loc)
    t = torch.stack([loc.real, loc.imag]).to(torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return complex(float(t[0]), float(t[1]))
