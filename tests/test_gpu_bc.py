"""GPU parity of the ghost-point faces (the mixed boundary conditions of the
Marmousi-II case of Sec. 4: sound-hard surface, first-order absorbing sides and
bottom) against the fp64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2506_03617_gb300 import inputs as I

from _parity import TOL_C128, TOL_LOW, TOL_OP, TOL_POINTWISE, TOL_SOLUTION, check, face_mask, pml_mask

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


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


CASES = [
    ("marmousi_2d", I.Grid(2, (150, 31), 0), I.MARMOUSI_BC),
    ("absorbing_pml_2d", I.Grid(2, (70, 44), 5), ("absorbing", "sound_hard", "dirichlet", "absorbing")),
    ("absorbing_3d", I.Grid(3, (21, 17, 13), 0),
     ("absorbing", "absorbing", "absorbing", "absorbing", "sound_hard", "absorbing")),
]


def _mask(grid):
    """PML cells and the boundary rows of the faces: the cells whose rows differ
    from the plain interior stencil."""
    return pml_mask(grid) | face_mask(grid)


def _pair(native, grid, bc, seed=41, **kw):
    c = I.marmousi_like(grid, seed) if grid.dim == 2 and grid.npml == 0 else \
        I.layered_grf(grid, seed=seed, corr_cells=4.0)
    p = I.paper_params(grid, c, ppw=10.0)
    P = oracle.Problem.from_grid(grid, c, p, bc=bc)
    G = native.Problem.from_grid(grid, c, p)
    G.set_boundary(bc)
    if kw:
        G.set_params(**kw)
    return P, G, c, p


@pytest.mark.parametrize("name,grid,bc", CASES)
@pytest.mark.parametrize("shifted", [False, True])
def test_operator_parity_with_faces(native, name, grid, bc, shifted):
    P, G, _, _ = _pair(native, grid, bc)
    x = I.random_complex(grid.n_total, 1)
    got = G.apply_operator(_cuda(x), shifted=shifted).cpu().numpy()
    check(got, P.apply(x, shifted=shifted), grid, TOL_OP, what=f"faces operator {name}", mask=_mask(grid))


@pytest.mark.parametrize("name,grid,bc", CASES)
@pytest.mark.parametrize("which", [0, 1, 2])
def test_phi_parity_with_faces_c128(native, name, grid, bc, which):
    P, G, _, _ = _pair(native, grid, bc, exp_tol=1e-12)
    x = I.random_complex(grid.n_total, 2)
    ref, _ = P.phi(which, x)
    got, _ = G.apply_phi(which, _cuda(x))
    check(got.cpu().numpy(), ref, grid, TOL_C128, what=f"faces phi{which} c128 {name}", mask=_mask(grid))


@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_low_precision_phi_with_faces(native, prec):
    """Faces run on the per-point sweep and on the persistent kernel (which adds
    the face term to the boundary rows after each step), never on the tiles."""
    grid, bc = CASES[0][1], CASES[0][2]
    P, G, _, _ = _pair(native, grid, bc, prec=prec, exp_tol=1e-6, persist_cfg=-2)
    assert G.tile_config()[0] == -1 and G.persist_config()[0] == -1
    x = I.random_complex(grid.n_total, 3)
    bound = TOL_LOW[prec]
    base = {}
    for which in (0, 1):
        ref, _ = P.phi(which, x)
        got, _ = G.apply_phi(which, _cuda(x))
        base[which] = got.cpu().numpy()
        check(base[which], ref, grid, TOL_POINTWISE[prec], what=f"faces per-point phi{which} {prec}",
              mask=_mask(grid))
    ran = set()
    for cfg in range(native.load().mxp_num_persist_configs()):
        G.set_params(persist_cfg=cfg)
        if G.persist_config()[0] != cfg:
            continue
        ran.add(cfg)
        assert G.tile_config()[0] == -1 and G.sweep_kernel() == "persistent_2d"
        for which in (0, 1):
            ref, _ = P.phi(which, x)
            got = G.apply_phi(which, _cuda(x))[0].cpu().numpy()
            check(got, ref, grid, bound, what=f"faces persist cfg {cfg} phi{which} {prec}", mask=_mask(grid))
            if prec == "c64":
                assert _rel(got, base[which]) < 5e-5, (cfg, which)
    # every configuration with face terms (all but the two face-free ones) ran
    assert ran == {0, 1, 2, 3, 4, 5, 8}, sorted(ran)


def test_matexpre_fixed_trip_parity_with_faces(native):
    grid, bc = CASES[0][1], CASES[0][2]
    P, G, _, _ = _pair(native, grid, bc, exp_tol=1e-12, inner_fixed=3)
    r = I.random_complex(grid.n_total, 4)
    ref, it, _ = P.matexpre(r, fixed=3)
    got, st = G.apply_matexpre(_cuda(r))
    assert st["inner_iters"] == it == 3
    check(got.cpu().numpy(), ref, grid, TOL_C128, what="faces matexpre fixed 3 c128", mask=_mask(grid))


def test_solve_parity_marmousi_like(native):
    """Sec. 4 Marmousi-II setting in miniature: source near the surface, centred
    in x; same outer count as the oracle, solution within 1e-8."""
    g, c, p = I.config_2d_marmousi_like(nx=80)
    P = oracle.Problem.from_grid(g, c, p, bc=I.MARMOUSI_BC)
    G = native.Problem.from_grid(g, c, p)
    G.set_boundary(I.MARMOUSI_BC)
    G.set_params(exp_tol=1e-12)
    b = I.rhs_from_source(I.gaussian_source(g, center=(0.5, 2.5 * g.h))).ravel()
    u_ref, info = P.fgmres(b, rtol=1e-6, maxit=300)
    x, st = G.solve(_cuda(b), rtol=1e-6, maxit=300)
    assert st["converged"] and info["converged"]
    assert st["outer_iters"] == info["outer_iters"]
    check(x.cpu().numpy(), u_ref, g, TOL_SOLUTION, what="faces solve marmousi-like c128", mask=_mask(g))


@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_low_precision_solve_with_faces_reaches_tolerance(native, prec):
    g, c, p = I.config_2d_marmousi_like(nx=300)
    P = oracle.Problem.from_grid(g, c, p, bc=I.MARMOUSI_BC)
    G = native.Problem.from_grid(g, c, p)
    G.set_boundary(I.MARMOUSI_BC)
    G.set_params(prec=prec, exp_tol=1e-6)
    b = I.rhs_from_source(I.gaussian_source(g, center=(0.5, 2.5 * g.h))).ravel()
    x, st = G.solve(_cuda(b), rtol=1e-6, maxit=300)
    assert st["converged"]
    assert np.linalg.norm(b - P.apply(x.cpu().numpy())) / np.linalg.norm(b) <= 1.000001e-6


def test_batch_with_faces(native):
    g, c, p = I.config_2d_marmousi_like(nx=80)
    P = oracle.Problem.from_grid(g, c, p, bc=I.MARMOUSI_BC)
    G = native.Problem.from_grid(g, c, p)
    G.set_boundary(I.MARMOUSI_BC)
    G.set_params(prec="c64", exp_tol=1e-6)
    srcs = [I.rhs_from_source(I.gaussian_source(g, center=(x0, 2.5 * g.h))).ravel()
            for x0 in (0.3, 0.5, 0.7)]
    bs = [_cuda(b) for b in srcs]
    xs = [G.empty() for _ in bs]
    stats = native.solve_batch([G], [0] * 3, bs, xs, rtol=1e-6, maxit=300)
    for b, x, st in zip(srcs, xs, stats):
        assert st["converged"]
        assert np.linalg.norm(b - P.apply(x.cpu().numpy())) / np.linalg.norm(b) <= 1.000001e-6


def test_boundary_arguments_are_checked_and_reversible(native):
    grid = I.Grid(2, (32, 16), 0)
    c = I.homogeneous(grid)
    p = I.paper_params(grid, c, ppw=10.0)
    G = native.Problem.from_grid(grid, c, p)
    with pytest.raises(native.MxpError):
        G.set_boundary([3, 0, 0, 0])
    with pytest.raises(native.MxpError):
        G.set_boundary([0, 0, 0, 0, 1, 0])            # z face of a 2D grid
    x = _cuda(I.random_complex(grid.n_total, 5))
    y0 = G.apply_operator(x).clone()
    G.set_boundary(I.MARMOUSI_BC)
    assert G.boundary() == (2, 2, 1, 2, 0, 0)
    assert not torch.equal(G.apply_operator(x), y0)
    G.set_boundary(None)
    assert torch.equal(G.apply_operator(x), y0)
