"""Multi-rank host logic on CPU with two gloo ranks: sharding covers every
source once, the job time is the slowest rank's and the work is summed."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2506_03617_gb300 import dist as D
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://")
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
