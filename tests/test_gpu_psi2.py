"""GPU parity of the psi_2 action and of the preconditioner on the second
inverse formula of Sec. 3.1 (r~ = psi_2(i t A_s) r, GMRES on
(I - psi_1(i t A_s)) w = r~) against the fp64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2506_03617_gb300 import inputs as I

from _parity import TOL_C128, TOL_C64, TOL_SOLUTION, check

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


def _setup(native, grid, seed=31, **kw):
    c = I.layered_grf(grid, seed=seed, corr_cells=4.0)
    p = I.paper_params(grid, c, ppw=10.0)
    P = oracle.Problem.from_grid(grid, c, p)
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(**kw)
    return P, G


@pytest.mark.parametrize("grid", [I.Grid(2, (290, 37), 5), I.Grid(3, (41, 29, 17), 3),
                                  I.Grid(2, (40, 36), 6)])
def test_psi2_action_parity_c128(native, grid):
    P, G = _setup(native, grid, exp_tol=1e-12)
    x = I.random_complex(grid.n_total, 2)
    ref, _ = P.phi(2, x)
    got, passes = G.apply_phi(2, _cuda(x))
    assert passes > 0
    check(got.cpu().numpy(), ref, grid, TOL_C128, what="psi2 c128")


@pytest.mark.parametrize("fuse_k", [0, 1])
def test_psi2_action_c64_fused_and_unfused(native, fuse_k):
    grid = I.Grid(2, (300, 260), 8)
    P, G = _setup(native, grid, prec="c64", exp_tol=1e-6, fuse_k=fuse_k)
    x = I.random_complex(grid.n_total, 5)
    ref, _ = P.phi(2, x)
    got, _ = G.apply_phi(2, _cuda(x))
    check(got.cpu().numpy(), ref, grid, TOL_C64, what=f"psi2 c64 fuse_k={fuse_k}")


def test_second_formula_fixed_trip_parity_c128(native):
    grid = I.Grid(2, (40, 36), 6)
    P, G = _setup(native, grid, exp_tol=1e-12, inner_fixed=3, precond=2)
    r = I.random_complex(grid.n_total, 3)
    ref, it, _ = P.matexpre(r, fixed=3, variant=1)
    got, st = G.apply_matexpre(_cuda(r))
    assert st["inner_iters"] == it == 3
    check(got.cpu().numpy(), ref, grid, TOL_C128, what="second formula fixed 3 c128")


def test_second_formula_tolerance_mode_matches_iterations(native):
    grid = I.Grid(2, (40, 36), 6)
    P, G = _setup(native, grid, exp_tol=1e-12, precond=2)
    r = I.random_complex(grid.n_total, 4)
    ref, it, _ = P.matexpre(r, fprtol=0.08, variant=1)
    got, st = G.apply_matexpre(_cuda(r))
    assert st["inner_iters"] == it
    check(got.cpu().numpy(), ref, grid, TOL_C128, what="second formula tolerance mode c128")


def test_second_formula_solve_parity(native):
    grid = I.Grid(2, (64, 64), 10)
    c = I.homogeneous(grid)
    p = I.paper_params(grid, c, ppw=10.0)
    P = oracle.Problem.from_grid(grid, c, p)
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(exp_tol=1e-12, precond=2)
    b = I.rhs_from_source(I.gaussian_source(grid)).ravel()
    u_ref, info = P.fgmres(b, rtol=1e-6, variant=1)
    x, st = G.solve(_cuda(b), rtol=1e-6)
    assert st["converged"] and info["converged"]
    assert st["outer_iters"] == info["outer_iters"]
    check(x.cpu().numpy(), u_ref, grid, TOL_SOLUTION, what="second formula solve c128")


@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_second_formula_low_precision_solve_reaches_tolerance(native, prec):
    grid = I.Grid(2, (128, 128), 16)
    c = I.layered_grf(grid, seed=33, corr_cells=6.0)
    p = I.paper_params(grid, c, ppw=10.0)
    P = oracle.Problem.from_grid(grid, c, p)
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec=prec, exp_tol=1e-6, precond=2)
    b = I.rhs_from_source(I.gaussian_source(grid)).ravel()
    x, st = G.solve(_cuda(b), rtol=1e-6, maxit=300)
    assert st["converged"]
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - P.apply(xh)) / np.linalg.norm(b) <= 1.000001e-6


def test_which_out_of_range_is_rejected(native):
    grid = I.Grid(2, (16, 16), 2)
    _, G = _setup(native, grid)
    x = _cuda(I.random_complex(grid.n_total, 1))
    with pytest.raises(native.MxpError):
        G.apply_phi(3, x)
    with pytest.raises(native.MxpError):
        G.set_params(precond=3)
