"""Multi-rank host logic on CPU with two gloo ranks: sharding covers every
source once, the job time is the slowest rank's and the work is summed, and a
multi-source solve split across the ranks (medium replicated, sources
round-robin, one gather at the end) returns exactly the one-rank results.  The
per-rank solver here is the oracle's FGMRES (on the GPU it is the batched
C-ABI solver); what is tested is the split and the gather."""
import os
import socket

import numpy as np
import pytest
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


# ---------------------------------------------------------------- slab decomposition

SLAB_GRID = I.Grid(2, (30, 40), 5)          # 40 x 50 unknowns: rows of 40 along y
SLAB_HALO = 3


def _slab_job():
    import oracle
    from paper_2506_03617_gb300 import native as N
    g = SLAB_GRID
    c = I.layered_grf(g, seed=I.SEED_BASE + 9200, corr_cells=3.0)
    p = I.paper_params(g, c, ppw=10.0)
    P = oracle.Problem.from_grid(g, c, p)
    x = I.random_complex(g.n_total, 77)
    S, m = N.taylor_plan(P.norm_inf_tA(True), 1e-12, 6.0, 1)      # host-only planner, shift mu = 0
    return P, p, x, (0.0, S, m)


def _oracle_slab_step(P, e0, e1):
    """out = rho (y + sigma A_s p) on rows [e0, e1) with zero values beyond them
    (what a slab problem's step computes, here through the oracle's operator)."""
    import torch
    g = SLAB_GRID
    row = g.n[0]

    def step(sigma, pv, yv, rho, out):
        full = np.zeros(g.n_total, dtype=np.complex128)
        full[e0 * row:e1 * row] = pv.numpy()
        ap = P.apply(full, shifted=True)[e0 * row:e1 * row]
        out.copy_(torch.from_numpy(rho * (yv.numpy() + sigma * ap)))
    return step


def _slab_worker(rank, world, port, q):
    import oracle
    import torch
    import torch.distributed as dist
    from paper_2506_03617_gb300 import dist as D
    _init(rank, world, port)
    oracle.set_threads(1)
    P, p, x, plan = _slab_job()
    g = SLAB_GRID
    rows, row = g.n[-1], g.n[0]
    bounds = D.slab_bounds(rows, world)
    e0, e1 = D.slab_extended(bounds, rank, SLAB_HALO, rows)
    r0, r1 = bounds[rank]
    p0 = torch.zeros((e1 - e0) * row, dtype=torch.complex128)
    p0[(r0 - e0) * row:(r1 - e0) * row] = torch.from_numpy(x[r0 * row:r1 * row])
    bufs = [torch.zeros_like(p0), torch.zeros_like(p0)]
    ex = D.SlabExchange(bounds, rank, SLAB_HALO, row, rows)
    res = D.slab_exp_action([_oracle_slab_step(P, e0, e1)], plan, p.t, [p0], [bufs], ex, SLAB_HALO)[0]
    owned = slice((r0 - e0) * row, (r1 - e0) * row)
    dot = D.slab_dot(res, res, owned)
    q.put((rank, r0, r1, res[owned].numpy().copy(), dot))
    dist.destroy_process_group()


def test_slab_decomposed_exp_action_matches_the_single_domain_oracle():
    """Two gloo ranks each hold half of the grid's rows plus 3 halo rows, run the
    sub-stepped Horner recurrence of exp(i t A_s) with a halo exchange every 3
    steps and at every sub-step end, and together reproduce the oracle's exp
    action on the whole grid; the allreduced dot equals the global one."""
    P, p, x, plan = _slab_job()
    ref = P.phi(0, x)[0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=600) for _ in range(2)), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    row = SLAB_GRID.n[0]
    got = np.zeros_like(ref)
    for _, r0, r1, vals, _ in out:
        got[r0 * row:r1 * row] = vals
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-10
    for *_, dot in out:
        assert abs(dot - np.vdot(got, got)) <= 1e-12 * abs(np.vdot(got, got))


def test_slab_bounds_cover_the_rows_once():
    from paper_2506_03617_gb300 import dist as D
    for n, w in ((50, 2), (51, 4), (7, 7)):
        b = D.slab_bounds(n, w)
        assert b[0][0] == 0 and b[-1][1] == n and all(b[k][1] == b[k + 1][0] for k in range(w - 1))
        assert max(r1 - r0 for r0, r1 in b) - min(r1 - r0 for r0, r1 in b) <= 1
    assert D.slab_extended(D.slab_bounds(50, 2), 0, 3, 50) == (0, 28)
    assert D.slab_extended(D.slab_bounds(50, 2), 1, 3, 50) == (22, 50)


# ------------------------------------------------- slab-decomposed FGMRES / Algorithm 1

SOLVE_GRID = I.Grid(2, (22, 26), 5)
SOLVE_HALO = 3


def _solve_job():
    import oracle
    from paper_2506_03617_gb300 import native as N
    g = SOLVE_GRID
    c = I.layered_grf(g, seed=I.SEED_BASE + 9400, corr_cells=3.0)
    p = I.paper_params(g, c, ppw=10.0, t_over_h2=10.0)
    P = oracle.Problem.from_grid(g, c, p)
    S, m = N.taylor_plan(P.norm_inf_tA(True), 1e-11, 6.0, 1)
    params = dict(t=p.t, fprtol=p.fprtol, inner_restart=30, inner_maxit=400, inner_fixed=0, precond=0,
                  neumann_n=0)
    b = I.rhs_from_source(I.gaussian_source(g)).ravel()
    return P, params, [(0.0, S, m)] * 3, b


def _run_slab_solve(world, rank, exchange, allreduce):
    import torch
    from _slab_oracle import OracleSlab
    from paper_2506_03617_gb300 import dist as D
    P, params, plans, b = _solve_job()
    g = SOLVE_GRID
    rows, row = g.n[-1], g.n[0]
    bounds = D.slab_bounds(rows, world)
    e0, e1 = D.slab_extended(bounds, rank, SOLVE_HALO, rows)
    r0, r1 = bounds[rank]
    slab = OracleSlab(P, g, e0, e1, params, plans)
    bs = torch.from_numpy(np.ascontiguousarray(b[e0 * row:e1 * row]))
    xs = torch.zeros_like(bs)
    solver = D.SlabSolver([slab], [(r0 - e0, r1 - e0)], exchange, allreduce, SOLVE_HALO)
    st = solver.solve([bs], [xs], rtol=1e-6, restart=30, maxit=60)
    return r0, r1, xs[(r0 - e0) * row:(r1 - e0) * row].numpy().copy(), st


def _slab_solve_worker(rank, world, port, q):
    import oracle
    import torch.distributed as dist
    from paper_2506_03617_gb300 import dist as D
    _init(rank, world, port)
    oracle.set_threads(1)
    bounds = D.slab_bounds(SOLVE_GRID.n[-1], world)
    ex = D.SlabExchange(bounds, rank, SOLVE_HALO, SOLVE_GRID.n[0], SOLVE_GRID.n[-1])
    q.put((rank,) + _run_slab_solve(world, rank, ex, D.torch_allreduce))
    dist.destroy_process_group()


def test_slab_decomposed_solve_matches_one_domain():
    """Algorithm 1 inside FGMRES(30) on a grid split into two slabs over gloo
    ranks (halo 3, every dot summed over the ranks) takes the same outer and
    inner iterations as the same driver on the whole grid, reaches the same
    solution, and meets rtol 1e-6 in the oracle's true residual."""
    import oracle
    P, _, _, b = _solve_job()
    oracle.set_threads(1)
    _, _, x1, st1 = _run_slab_solve(1, 0, lambda vs: None, None)
    assert st1["converged"] and st1["outer_iters"] > 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_solve_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=900) for _ in range(2)), key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    row = SOLVE_GRID.n[0]
    x2 = np.zeros_like(x1)
    for _, r0, r1, vals, st in out:
        x2[r0 * row:r1 * row] = vals
        assert (st["outer_iters"], st["inner_iters_total"]) == (st1["outer_iters"], st1["inner_iters_total"])
    assert np.linalg.norm(x2 - x1) / np.linalg.norm(x1) < 1e-9
    assert np.linalg.norm(b - P.apply(x2)) / np.linalg.norm(b) <= 1.000001e-6


def test_slab_least_squares_matches_numpy():
    """The host least squares of the slab solver (Givens rotations applied
    column by column to the (R + 1) x R Hessenberg matrix): residual estimates
    and solutions equal numpy's least-squares solution of min ||beta e1 - H y||
    for every leading size."""
    from paper_2506_03617_gb300 import dist as D
    rng = np.random.default_rng(5)
    R = 12
    H = np.triu(rng.standard_normal((R + 1, R)) + 1j * rng.standard_normal((R + 1, R)), -1)
    beta = 2.5
    lsq = D._Lsq(R, beta)
    for j in range(R):
        est = lsq.add(j, H[:j + 1, j], H[j + 1, j])
        e1 = np.zeros(j + 2, dtype=np.complex128)
        e1[0] = beta
        y_ref = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
        res_ref = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y_ref)
        assert abs(est - res_ref) <= 1e-12 * beta
        assert np.max(np.abs(lsq.solve(j + 1) - y_ref)) <= 1e-10 * np.max(np.abs(y_ref))


def test_givens_zeroes_the_second_entry():
    from paper_2506_03617_gb300 import dist as D
    for a, b in [(1 + 2j, 3 - 1j), (0j, 2 + 1j), (1.5 + 0j, 0j), (-2j, 1e-3 + 4j)]:
        c, s = D._givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        v = G @ np.array([a, b])
        assert abs(v[1]) <= 1e-14 * (abs(a) + abs(b))
        assert abs(abs(v[0]) - np.hypot(abs(a), abs(b))) <= 1e-14 * (abs(a) + abs(b))
        assert np.allclose(G.conj().T @ G, np.eye(2), atol=1e-14)


@pytest.mark.parametrize("which,world,halo", [(0, 2, 2), (1, 3, 4), (2, 2, 3)])
def test_slab_phi_actions_match_the_oracle(which, world, halo):
    """exp, psi_1 and psi_2 actions of the slab driver (augmented scalar rows for
    the psi actions, halo exchange every `halo` Horner steps) on slabs of one
    grid held by one process, against the oracle's actions on the whole grid."""
    import torch
    import oracle
    from _slab_oracle import OracleSlab
    from paper_2506_03617_gb300 import dist as D
    from paper_2506_03617_gb300 import native as N
    g = I.Grid(2, (18, 22), 4)
    c = I.layered_grf(g, seed=I.SEED_BASE + 9600, corr_cells=3.0)
    p = I.paper_params(g, c, ppw=10.0, t_over_h2=10.0)
    P = oracle.Problem.from_grid(g, c, p)
    S, m = N.taylor_plan(1.2 * P.norm_inf_tA(True), 1e-14, 4.0, 1)   # margin for the augmented rows
    params = dict(t=p.t, fprtol=p.fprtol, inner_restart=30, inner_maxit=100, inner_fixed=0, precond=0,
                  neumann_n=0)
    rows, row = g.n[-1], g.n[0]
    bounds = D.slab_bounds(rows, world)
    ext = [D.slab_extended(bounds, k, halo, rows) for k in range(world)]
    slabs = [OracleSlab(P, g, e0, e1, params, [(0.0, S, m)] * 3) for e0, e1 in ext]
    x = I.random_complex(g.n_total, 33)
    xs = [torch.from_numpy(np.ascontiguousarray(x[e0 * row:e1 * row])) for e0, e1 in ext]
    outs = [torch.zeros_like(v) for v in xs]
    solver = D.SlabSolver(slabs, [(r0 - e0, r1 - e0) for (e0, _), (r0, r1) in zip(ext, bounds)],
                          D.LocalSlabExchange(bounds, halo, row, rows), None, halo)
    solver.phi(which, xs, outs)
    got = np.zeros_like(x)
    for (e0, _), (r0, r1), v in zip(ext, bounds, outs):
        got[r0 * row:r1 * row] = v.numpy()[(r0 - e0) * row:(r1 - e0) * row]
    ref = P.phi(which, x)[0]
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-10


@pytest.mark.parametrize("precond", [1, 2])
def test_slab_solver_other_preconditioners_match_one_domain(precond):
    """The slab driver with the truncated Neumann series (precond 1, N = 2) and
    with the second inverse formula (precond 2) on three CPU slabs in one process
    takes the one-domain run's iteration counts and solution, and meets rtol in
    the oracle's true residual."""
    import torch
    import oracle
    from _slab_oracle import OracleSlab
    from paper_2506_03617_gb300 import dist as D
    from paper_2506_03617_gb300 import native as N
    g = I.Grid(2, (16, 20), 4)
    c = I.layered_grf(g, seed=I.SEED_BASE + 9700, corr_cells=3.0)
    p = I.paper_params(g, c, ppw=10.0, t_over_h2=10.0)
    P = oracle.Problem.from_grid(g, c, p)
    S, m = N.taylor_plan(1.2 * P.norm_inf_tA(True), 1e-12, 4.0, 1)
    params = dict(t=p.t, fprtol=p.fprtol, inner_restart=30, inner_maxit=200, inner_fixed=0, precond=precond,
                  neumann_n=2)
    b = I.rhs_from_source(I.gaussian_source(g)).ravel()
    rows, row = g.n[-1], g.n[0]

    def run(world, halo):
        bounds = D.slab_bounds(rows, world)
        ext = [D.slab_extended(bounds, k, halo, rows) for k in range(world)]
        slabs = [OracleSlab(P, g, e0, e1, params, [(0.0, S, m)] * 3) for e0, e1 in ext]
        bs = [torch.from_numpy(np.ascontiguousarray(b[e0 * row:e1 * row])) for e0, e1 in ext]
        xs = [torch.zeros_like(v) for v in bs]
        ex = D.LocalSlabExchange(bounds, halo, row, rows) if world > 1 else (lambda vs: None)
        solver = D.SlabSolver(slabs, [(r0 - e0, r1 - e0) for (e0, _), (r0, r1) in zip(ext, bounds)], ex, None,
                              halo)
        st = solver.solve(bs, xs, rtol=1e-6, restart=30, maxit=80)
        x = np.zeros_like(b)
        for (e0, _), (r0, r1), v in zip(ext, bounds, xs):
            x[r0 * row:r1 * row] = v.numpy()[(r0 - e0) * row:(r1 - e0) * row]
        return x, st

    x1, st1 = run(1, 3)
    x3, st3 = run(3, 3)
    assert st1["converged"] and st3["converged"]
    assert (st3["outer_iters"], st3["inner_iters_total"]) == (st1["outer_iters"], st1["inner_iters_total"])
    assert np.linalg.norm(x3 - x1) / np.linalg.norm(x1) < 1e-9
    assert np.linalg.norm(b - P.apply(x3)) / np.linalg.norm(b) <= 1.000001e-6
