"""Batched solves (several sources per medium advancing in lockstep, one sweep
launch per pass for the whole batch, sweep sequences replayed from captured
CUDA graphs): every right-hand side reaches the 1e-6 true residual (checked
with the oracle's operator) and matches its single-source solve; in complex128
the first source of each medium also takes the oracle's outer iteration count
and its solution agrees with the oracle's element-wise within 1e-8."""
import numpy as np
import pytest

import oracle
from paper_2506_03617_gb300 import inputs as I

from _parity import TOL_SOLUTION, check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03617_gb300 import native as N
    N.load()
    return N


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_batch_of_sources_on_two_media(native, prec):
    grids = [I.Grid(2, (96, 80), 10), I.Grid(2, (64, 64), 8)]
    probs, oracles, srcs = [], [], []
    for k, g in enumerate(grids):
        c = I.layered_grf(g, seed=I.SEED_BASE + 4000 + k, corr_cells=4.0)
        p = I.paper_params(g, c, ppw=10.0)
        G = native.Problem.from_grid(g, c, p)
        G.set_params(prec=prec, exp_tol=1e-6 if prec == "c64" else 1e-12)
        probs.append(G)
        oracles.append(oracle.Problem.from_grid(g, c, p))
        for ctr in I.random_centers(g, 3, seed=I.SEED_BASE + 4100 + k):
            srcs.append((k, I.rhs_from_source(I.gaussian_source(g, center=ctr)).ravel()))
    bs = [torch.from_numpy(b).cuda() for _, b in srcs]
    xs = [probs[k].empty() for k, _ in srcs]
    stats = native.solve_batch(probs, [k for k, _ in srcs], bs, xs, rtol=1e-6, maxit=100)
    seen = set()
    for (k, b), x, st in zip(srcs, xs, stats):
        assert st["converged"], st
        xh = x.cpu().numpy()
        assert np.linalg.norm(b - oracles[k].apply(xh)) / np.linalg.norm(b) <= 1.000001e-6
        # agrees with the single-source path to the solve tolerance
        x1, _ = probs[k].solve(torch.from_numpy(b).cuda(), rtol=1e-6)
        assert _rel(xh, x1.cpu().numpy()) < 1e-4
        if prec == "c128" and k not in seen:
            # the oracle's Algorithm 1 + FGMRES on the same source
            seen.add(k)
            u_ref, info = oracles[k].fgmres(b, rtol=1e-6)
            assert st["outer_iters"] == info["outer_iters"], (st["outer_iters"], info["outer_iters"])
            check(xh, u_ref, grids[k], TOL_SOLUTION, what=f"batched solve c128 medium {k}")


def test_batch_is_repeatable_with_replayed_graphs(native):
    g = I.Grid(2, (64, 64), 8)
    c = I.homogeneous(g)
    p = I.paper_params(g, c, ppw=10.0)
    G = native.Problem.from_grid(g, c, p)
    G.set_params(prec="c64", exp_tol=1e-6)
    bs = [torch.from_numpy(I.rhs_from_source(I.gaussian_source(g, center=ctr)).ravel()).cuda()
          for ctr in I.random_centers(g, 4, seed=7)]
    x1 = [G.empty() for _ in bs]
    x2 = [G.empty() for _ in bs]
    native.solve_batch([G], [0] * 4, bs, x1)
    native.solve_batch([G], [0] * 4, bs, x2)          # second call replays captured graphs
    for a, b in zip(x1, x2):
        assert torch.equal(a, b)


def test_uneven_problems_solve_concurrently_on_their_own_streams(native):
    """Problems of different grid sizes in one call run in their own host
    threads; each uses the stream it was created on."""
    grids = [I.Grid(2, (160, 144), 12), I.Grid(2, (72, 64), 8)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    probs, oracles, srcs = [], [], []
    for k, (g, s) in enumerate(zip(grids, streams)):
        c = I.layered_grf(g, seed=I.SEED_BASE + 4200 + k, corr_cells=4.0)
        p = I.paper_params(g, c, ppw=10.0)
        G = native.Problem.from_grid(g, c, p, stream=s)
        G.set_params(prec="c64", exp_tol=1e-6)
        probs.append(G)
        oracles.append(oracle.Problem.from_grid(g, c, p))
        for ctr in I.random_centers(g, 2, seed=I.SEED_BASE + 4300 + k):
            srcs.append((k, I.rhs_from_source(I.gaussian_source(g, center=ctr)).ravel()))
    srcs = [srcs[2], srcs[0], srcs[1], srcs[3]]       # right-hand sides interleaved across problems
    bs = [torch.from_numpy(b).cuda() for _, b in srcs]
    xs = [probs[k].empty() for k, _ in srcs]
    torch.cuda.synchronize()
    stats = native.solve_batch(probs, [k for k, _ in srcs], bs, xs, rtol=1e-6, maxit=100)
    torch.cuda.synchronize()
    for (k, b), x, st in zip(srcs, xs, stats):
        assert st["converged"], st
        xh = x.cpu().numpy()
        assert np.linalg.norm(b - oracles[k].apply(xh)) / np.linalg.norm(b) <= 1.000001e-6
    # each problem alone gives the same solutions to the solve tolerance
    for k in range(2):
        mine = [i for i, (kk, _) in enumerate(srcs) if kk == k]
        xs1 = [probs[k].empty() for _ in mine]
        native.solve_batch([probs[k]], [0] * len(mine), [bs[i] for i in mine], xs1, rtol=1e-6,
                           maxit=100)
        torch.cuda.synchronize()
        for i, x1 in zip(mine, xs1):
            assert _rel(xs[i].cpu().numpy(), x1.cpu().numpy()) < 1e-4


@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_grouped_solve_of_mixed_grid_sizes(native, prec):
    """Three media of different grid sizes in one mxp_solve_batch call form one
    group: every pass of every action is one launch over all (problem, source,
    tile) items, converged sources are switched off by a device mask.  Each
    source reaches the 1e-6 true residual of the oracle's operator, the first
    source of each medium agrees with the oracle's FP64 solution within 1e-5,
    every source agrees with its problem solved alone, and the group needs far
    fewer kernel launches than the problems one after another."""
    grids = [I.Grid(2, (96, 80), 10), I.Grid(2, (64, 64), 8), I.Grid(2, (48, 40), 6)]
    probs, oracles, srcs = [], [], []
    for k, g in enumerate(grids):
        c = I.layered_grf(g, seed=I.SEED_BASE + 4400 + k, corr_cells=4.0)
        p = I.paper_params(g, c, ppw=10.0)
        G = native.Problem.from_grid(g, c, p)
        G.set_params(prec=prec, exp_tol=1e-6)
        probs.append(G)
        oracles.append(oracle.Problem.from_grid(g, c, p))
        for ctr in I.random_centers(g, 3, seed=I.SEED_BASE + 4500 + k):
            srcs.append((k, I.rhs_from_source(I.gaussian_source(g, center=ctr)).ravel()))
    order = [3, 0, 6, 1, 4, 7, 2, 5, 8]                 # interleaved across problems
    srcs = [srcs[i] for i in order]
    bs = [torch.from_numpy(b).cuda() for _, b in srcs]
    xs = [probs[k].empty() for k, _ in srcs]
    l0 = native.kernel_launch_count()
    stats = native.solve_batch(probs, [k for k, _ in srcs], bs, xs, rtol=1e-6, maxit=100)
    torch.cuda.synchronize()
    grouped_launches = native.kernel_launch_count() - l0
    seen = set()
    for (k, b), x, st in zip(srcs, xs, stats):
        assert st["converged"], st
        assert st["seconds"] > 0 and st["stencil_passes"] > 0
        xh = x.cpu().numpy()
        assert np.linalg.norm(b - oracles[k].apply(xh)) / np.linalg.norm(b) <= 1.000001e-6
        if k not in seen:
            seen.add(k)
            u_ref, _ = oracles[k].fgmres(b, rtol=1e-6)
            check(xh, u_ref, grids[k], 1e-5, what=f"grouped solve {prec} medium {k}")
    # each problem alone (the single-problem lockstep path)
    alone = 0
    for k in range(3):
        mine = [i for i, (kk, _) in enumerate(srcs) if kk == k]
        xs1 = [probs[k].empty() for _ in mine]
        l1 = native.kernel_launch_count()
        native.solve_batch([probs[k]], [0] * len(mine), [bs[i] for i in mine], xs1, rtol=1e-6, maxit=100)
        torch.cuda.synchronize()
        alone += native.kernel_launch_count() - l1
        for i, x1 in zip(mine, xs1):
            assert _rel(xs[i].cpu().numpy(), x1.cpu().numpy()) < 1e-4
    assert grouped_launches < 0.8 * alone, (grouped_launches, alone)


def test_large_problem_in_a_batch_solves_its_sources_one_by_one(native):
    """A 2D problem on the persistent kernel with at least 2^20 unknowns (the
    1088^2 layered workload) solves its sources one after another inside
    mxp_solve_batch, while a small problem in the same call keeps the lockstep
    path: each large source gives exactly its single-source solve (same outer
    and inner counts, same solution), and every source meets the oracle's true
    residual."""
    g, c, p = I.config_2d_layered()
    G = native.Problem.from_grid(g, c, p)
    G.set_params(prec="c64", exp_tol=1e-3, theta_max=6.0)
    assert G.persist_config()[0] >= 0 and g.n_total >= 1 << 20
    gs = I.Grid(2, (64, 64), 8)
    cs = I.layered_grf(gs, seed=I.SEED_BASE + 4600, corr_cells=4.0)
    ps = I.paper_params(gs, cs, ppw=10.0)
    Gs = native.Problem.from_grid(gs, cs, ps)
    Gs.set_params(prec="c64", exp_tol=1e-6)
    big = [I.rhs_from_source(I.gaussian_source(g, center=ctr)).ravel()
           for ctr in I.random_centers(g, 2, seed=I.SEED_BASE + 4610)]
    small = [I.rhs_from_source(I.gaussian_source(gs, center=ctr)).ravel()
             for ctr in I.random_centers(gs, 2, seed=I.SEED_BASE + 4620)]
    bs = [torch.from_numpy(b).cuda() for b in big + small]
    xs = [G.empty(), G.empty(), Gs.empty(), Gs.empty()]
    stats = native.solve_batch([G, Gs], [0, 0, 1, 1], bs, xs, rtol=1e-6, maxit=300)
    torch.cuda.synchronize()
    P = oracle.Problem.from_grid(g, c, p)
    Ps = oracle.Problem.from_grid(gs, cs, ps)
    for i, b in enumerate(big):
        x1, st1 = G.solve(bs[i], rtol=1e-6, maxit=300)
        assert (stats[i]["outer_iters"], stats[i]["inner_iters_total"]) == (st1["outer_iters"], st1["inner_iters_total"])
        xh = xs[i].cpu().numpy()
        assert _rel(xh, x1.cpu().numpy()) < 1e-12
        assert np.linalg.norm(b - P.apply(xh)) / np.linalg.norm(b) <= 1.000001e-6
    for i, b in enumerate(small):
        assert stats[2 + i]["converged"]
        xh = xs[2 + i].cpu().numpy()
        assert np.linalg.norm(b - Ps.apply(xh)) / np.linalg.norm(b) <= 1.000001e-6
