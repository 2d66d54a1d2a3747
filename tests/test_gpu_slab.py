"""Slab decomposition on one GPU: the rows of one grid split into slabs with
halo rows (the distributed layout of Sec. 4), each slab a problem of its own
(mxp_create_slab) stepped by mxp_horner_step, the halos refreshed by copies
between the slabs.  The owned rows reproduce the single-domain exp action of
the GPU path and of the fp64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2506_03617_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03617_gb300 import native as N
    N.load()
    return N


def _slabs(N, grid, c, params, world, halo):
    from paper_2506_03617_gb300 import dist as D
    rows, row = grid.n[-1], int(np.prod(grid.n[:-1]))
    bounds = D.slab_bounds(rows, world)
    cr = (float(c.min()), float(c.max()))
    cf = np.asarray(c).reshape(-1)
    probs = []
    for k in range(world):
        e0, e1 = D.slab_extended(bounds, k, halo, rows)
        S = N.Problem.slab(grid, e0, e1 - e0, cf[e0 * row:e1 * row], cr, params)
        S.set_params(exp_tol=1e-12)
        probs.append((S, e0, e1))
    return bounds, probs, row


@pytest.mark.parametrize("dim,world,halo", [(2, 2, 3), (2, 3, 4), (3, 2, 2)])
def test_slab_exp_action_matches_single_domain(native, dim, world, halo):
    from paper_2506_03617_gb300 import dist as D
    if dim == 2:
        g = I.Grid(2, (40, 52), 6)
        c = I.layered_grf(g, seed=I.SEED_BASE + 9300, corr_cells=4.0)
    else:
        g = I.Grid(3, (14, 12, 18), 4)
        c = I.layered_grf(g, seed=I.SEED_BASE + 9301, corr_cells=3.0)
    p = I.paper_params(g, c, ppw=10.0)
    x = I.random_complex(g.n_total, 91)
    G = native.Problem.from_grid(g, c, p)
    G.set_params(exp_tol=1e-12)
    bounds, probs, row = _slabs(native, g, c, p, world, halo)
    plan = G.plan(0)
    for S, _, _ in probs:
        assert S.plan(0) == plan            # every slab takes the whole grid's mu, S, m
    xd = torch.from_numpy(x).cuda()
    p0s, bufs, steps = [], [], []
    for (S, e0, e1), (r0, r1) in zip(probs, bounds):
        v = torch.zeros((e1 - e0) * row, dtype=torch.complex128, device="cuda")
        v[(r0 - e0) * row:(r1 - e0) * row] = xd[r0 * row:r1 * row]
        p0s.append(v)
        bufs.append([torch.zeros_like(v), torch.zeros_like(v)])
        steps.append(lambda sigma, pv, yv, rho, out, S=S: S.horner_step(sigma, pv, yv, rho=rho, out=out))
    ex = D.LocalSlabExchange(bounds, halo, row, g.n[-1])
    res = D.slab_exp_action(steps, plan, p.t, p0s, bufs, ex, halo)
    torch.cuda.synchronize()
    got = torch.empty_like(xd)
    for (S, e0, e1), (r0, r1), v in zip(probs, bounds, res):
        got[r0 * row:r1 * row] = v[(r0 - e0) * row:(r1 - e0) * row]
    single, _ = G.apply_phi(0, xd)
    ref = oracle.Problem.from_grid(g, c, p).phi(0, x)[0]
    scale = float(np.max(np.abs(ref)))
    got_h, single_h = got.cpu().numpy(), single.cpu().numpy()
    assert np.max(np.abs(got_h - ref)) / scale < 1e-10
    assert np.max(np.abs(got_h - single_h)) / scale < 1e-10
    # the distributed dot of the slab results equals the global one
    d = sum(D.slab_dot(v, v, slice((r0 - e0) * row, (r1 - e0) * row)) for (S, e0, e1), (r0, r1), v
            in zip(probs, bounds, res))
    assert abs(d - np.vdot(got_h, got_h)) <= 1e-12 * abs(np.vdot(got_h, got_h))


def test_slab_refuses_whole_grid_calls(native):
    g = I.Grid(2, (20, 24), 4)
    c = np.ones(g.n_total)
    p = I.paper_params(g, c)
    row = g.n[0]
    S = native.Problem.slab(g, 5, 10, c[5 * row:15 * row], (1.0, 1.0), p)
    x = torch.zeros(S.n_total, dtype=torch.complex128, device="cuda")
    with pytest.raises(native.MxpError):
        S.apply_phi(0, x)
    with pytest.raises(native.MxpError):
        native.Problem.slab(g, 20, 20, c[:20 * row], (1.0, 1.0), p)      # rows beyond the grid
    with pytest.raises(native.MxpError):
        native.Problem.slab(g, 0, 10, 2 * c[:10 * row], (1.0, 1.5), p)   # range misses the slab's speeds


@pytest.mark.parametrize("world,halo", [(2, 3), (3, 2)])
def test_slab_decomposed_solve_matches_single_domain(native, world, halo):
    """Algorithm 1 inside FGMRES(30) with the grid in slabs (SlabSolver: slab
    problems, halo copies between them, dots summed over the slabs) against the
    library's single-domain complex128 solve: the same outer and inner
    iteration counts, the same solution to 1e-8, and the oracle's true residual
    at rtol."""
    from paper_2506_03617_gb300 import dist as D
    g = I.Grid(2, (48, 40), 8)
    c = I.layered_grf(g, seed=I.SEED_BASE + 9500, corr_cells=4.0)
    p = I.paper_params(g, c, ppw=10.0)
    b = I.rhs_from_source(I.gaussian_source(g)).ravel()
    G = native.Problem.from_grid(g, c, p)
    G.set_params(prec="c128", exp_tol=1e-12)
    x_ref, st_ref = G.solve(torch.from_numpy(b).cuda(), rtol=1e-6)
    bounds, probs, row = _slabs(native, g, c, p, world, halo)
    slabs = [S for S, _, _ in probs]
    owned = [(r0 - e0, r1 - e0) for (S, e0, e1), (r0, r1) in zip(probs, bounds)]
    bd = torch.from_numpy(b).cuda()
    bs = [bd[e0 * row:e1 * row].clone() for _, e0, e1 in probs]
    xs = [torch.zeros_like(v) for v in bs]
    solver = D.SlabSolver(slabs, owned, D.LocalSlabExchange(bounds, halo, row, g.n[-1]), None, halo)
    st = solver.solve(bs, xs, rtol=1e-6, restart=30, maxit=300)
    torch.cuda.synchronize()
    x = torch.empty_like(bd)
    for (S, e0, e1), (r0, r1), v in zip(probs, bounds, xs):
        x[r0 * row:r1 * row] = v[(r0 - e0) * row:(r1 - e0) * row]
    assert st["converged"]
    assert (st["outer_iters"], st["inner_iters_total"]) == (st_ref["outer_iters"], st_ref["inner_iters_total"])
    xh, xr = x.cpu().numpy(), x_ref.cpu().numpy()
    assert np.linalg.norm(xh - xr) / np.linalg.norm(xr) < 1e-8
    P = oracle.Problem.from_grid(g, c, p)
    assert np.linalg.norm(b - P.apply(xh)) / np.linalg.norm(b) <= 1.000001e-6
