"""Multi-rank host logic on CPU with two gloo ranks: sharding covers every
source once, the job time is the slowest rank's and the work is summed, and a
multi-source solve split across the ranks (medium replicated, sources
round-robin, one gather at the end) returns exactly the one-rank results.  The
per-rank solver here is the oracle's FGMRES (on the GPU it is the batched
C-ABI solver); what is tested is the split and the gather."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2506_03617_gb300 import inputs as I


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://")


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2506_03617_gb300 import dist as D
    _init(rank, world, port)
    r, w, lr = D.env()
    mine = D.shard(range(10), r, w)
    D.barrier()
    t, u = D.reduce_job(seconds=1.0 + r, units=len(mine))
    q.put((r, mine, t, u))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    assert sorted(out[0][1] + out[1][1]) == list(range(10))
    for r, mine, t, u in out:
        assert t == 2.0 and u == 10.0


def test_single_process_is_the_identity():
    from paper_2506_03617_gb300 import dist as D
    assert D.reduce_job(3.5, 7) == (3.5, 7.0)
    assert D.shard([1, 2, 3], 0, 1) == [1, 2, 3]


# ---------------------------------------------------------------- sharded solves

GRID = I.Grid(2, (24, 20), 4)
NSRC = 5


def _job():
    c = I.layered_grf(GRID, seed=I.SEED_BASE + 9100, corr_cells=3.0)
    p = I.paper_params(GRID, c, ppw=10.0)
    centers = I.random_centers(GRID, NSRC, seed=I.SEED_BASE + 9101)
    srcs = [I.rhs_from_source(I.gaussian_source(GRID, center=ctr)).ravel() for ctr in centers]
    return c, p, srcs


def _solve_share_with_oracle(c, p, log=None):
    import oracle
    oracle.set_threads(1)
    P = oracle.Problem.from_grid(GRID, c, p)

    def solve_share(share):
        out = []
        for i, b in share:
            if log is not None:
                log.append(i)
            u, info = P.fgmres(b, rtol=1e-6)
            out.append({"x": u, "outer": info["outer_iters"], "converged": info["converged"]})
        return out
    return solve_share


def _sharded_worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2506_03617_gb300 import dist as D
    _init(rank, world, port)
    c, p, srcs = _job()
    log = []
    res = D.solve_sharded(srcs, _solve_share_with_oracle(c, p, log))
    q.put((rank, log, [(r["outer"], r["x"]) for r in res]))
    dist.destroy_process_group()


def test_sources_split_over_two_ranks_match_one_rank():
    from paper_2506_03617_gb300 import dist as D
    c, p, srcs = _job()
    ref = D.solve_sharded(srcs, _solve_share_with_oracle(c, p), rank=0, world=1)
    assert all(r["converged"] for r in ref)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted(q.get(timeout=300) for _ in range(2))
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    # each source solved by exactly one rank: 0, 2, 4 on rank 0 and 1, 3 on rank 1
    assert out[0][1] == [0, 2, 4] and out[1][1] == [1, 3]
    for _, _, res in out:                     # every rank receives every result
        assert len(res) == NSRC
        for (outer, x), r in zip(res, ref):
            assert outer == r["outer"]
            assert np.array_equal(x, r["x"])


def test_gather_rejects_missing_and_duplicate_units():
    import pytest
    from paper_2506_03617_gb300 import dist as D
    with pytest.raises(RuntimeError):
        D.gather_by_index({0: 1, 2: 3}, 3)
    with pytest.raises(RuntimeError):
        D.gather_by_index({5: 1}, 3)
    assert D.gather_by_index({1: "b", 0: "a"}, 2) == ["a", "b"]
