"""GPU parity: the CUDA path (through the C ABI) against the fp64 oracle.

Tolerances: 1e-10 relative per operator / exp / psi_1 / MatExPre application in
complex128 with the inner iteration count fixed, 1e-8 on the final solution;
complex64 and bfloat16-storage errors are measured and bounded."""
import math

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


def _pair(native, grid, c, params, **kw):
    P = oracle.Problem.from_grid(grid, c, params)
    G = native.Problem.from_grid(grid, c, params)
    if kw:
        G.set_params(**kw)
    return P, G


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


CASES = [
    ("2d_ragged", I.Grid(2, (290, 37), 5), "grf"),       # 300 x 47: three 128-wide blocks, ragged tail
    ("3d_ragged", I.Grid(3, (41, 29, 17), 3), "grf"),
    ("2d_nopml", I.Grid(2, (64, 50), 0), "one"),
    ("3d_thin", I.Grid(3, (1, 5, 9), 2), "one"),          # degenerate axis of one interior cell
]


def _medium(grid, kind, seed=21):
    if kind == "one":
        return I.homogeneous(grid)
    return I.layered_grf(grid, seed=seed, corr_cells=4.0)


@pytest.mark.parametrize("name,grid,kind", CASES)
@pytest.mark.parametrize("shifted", [False, True])
def test_operator_parity(native, name, grid, kind, shifted):
    c = _medium(grid, kind)
    p = I.paper_params(grid, c, ppw=10.0)
    P, G = _pair(native, grid, c, p)
    x = I.random_complex(grid.n_total, 1)
    ref = P.apply(x, shifted=shifted)
    got = G.apply_operator(_cuda(x), shifted=shifted).cpu().numpy()
    assert _rel(got, ref) < 1e-13


@pytest.mark.parametrize("name,grid,kind", CASES[:2] + [("2d_small", I.Grid(2, (40, 36), 6), "grf")])
@pytest.mark.parametrize("which", [0, 1])
def test_phi_parity_c128(native, name, grid, kind, which):
    c = _medium(grid, kind)
    p = I.paper_params(grid, c, ppw=10.0)
    P, G = _pair(native, grid, c, p, exp_tol=1e-12)
    x = I.random_complex(grid.n_total, 2)
    ref = P.phi(which, x)[0]
    got, passes = G.apply_phi(which, _cuda(x))
    assert passes > 0
    assert _rel(got.cpu().numpy(), ref) < 1e-10


def test_matexpre_fixed_trip_parity_c128(native):
    grid = I.Grid(2, (40, 36), 6)
    c = _medium(grid, "grf")
    p = I.paper_params(grid, c, ppw=10.0)
    P, G = _pair(native, grid, c, p, exp_tol=1e-12, inner_fixed=3)
    r = I.random_complex(grid.n_total, 3)
    ref, it, _ = P.matexpre(r, fixed=3)
    got, st = G.apply_matexpre(_cuda(r))
    assert st["inner_iters"] == it == 3
    assert _rel(got.cpu().numpy(), ref) < 1e-10


def test_matexpre_tolerance_mode_matches_iterations(native):
    grid = I.Grid(2, (40, 36), 6)
    c = _medium(grid, "grf")
    p = I.paper_params(grid, c, ppw=10.0)
    P, G = _pair(native, grid, c, p, exp_tol=1e-12)
    r = I.random_complex(grid.n_total, 4)
    ref, it, _ = P.matexpre(r, fprtol=0.08)
    got, st = G.apply_matexpre(_cuda(r))
    assert st["inner_iters"] == it
    assert _rel(got.cpu().numpy(), ref) < 1e-10


def test_solve_parity_2d_homogeneous_small(native):
    """FGMRES(30) + Algorithm 1 to 1e-6 on a 2D homogeneous grid with a Gaussian
    source at the centre: same outer count, solutions within 1e-8."""
    grid = I.Grid(2, (64, 64), 10)
    c = I.homogeneous(grid)
    p = I.paper_params(grid, c, ppw=10.0)
    P, G = _pair(native, grid, c, p, exp_tol=1e-12)
    b = I.rhs_from_source(I.gaussian_source(grid)).ravel()
    u_ref, info = P.fgmres(b, rtol=1e-6)
    x, st = G.solve(_cuda(b), rtol=1e-6)
    assert st["converged"] and info["converged"]
    assert st["outer_iters"] == info["outer_iters"]
    assert _rel(x.cpu().numpy(), u_ref) < 1e-8


@pytest.mark.parametrize("prec,bound", [("c64", 2e-4), ("bf16s", 8e-2)])
def test_low_precision_phi_error_bounded(native, prec, bound):
    grid = I.Grid(2, (40, 36), 6)
    c = _medium(grid, "grf")
    p = I.paper_params(grid, c, ppw=10.0)
    P, G = _pair(native, grid, c, p, prec=prec, exp_tol=1e-6)
    x = I.random_complex(grid.n_total, 5)
    for which in (0, 1):
        ref = P.phi(which, x)[0]
        got = G.apply_phi(which, _cuda(x))[0].cpu().numpy()
        assert _rel(got, ref) < bound, (prec, which, _rel(got, ref))


@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_low_precision_solve_reaches_fp64_tolerance(native, prec):
    """Pattern (1): a low-precision MatExPre inside fp64 FGMRES still reaches the
    1e-6 true residual; its error against the fp64 oracle solution is bounded."""
    grid = I.Grid(2, (64, 64), 10)
    c = I.homogeneous(grid)
    p = I.paper_params(grid, c, ppw=10.0)
    P, G = _pair(native, grid, c, p, prec=prec, exp_tol=1e-6)
    b = I.rhs_from_source(I.gaussian_source(grid)).ravel()
    u_ref, _ = P.fgmres(b, rtol=1e-6)
    x, st = G.solve(_cuda(b), rtol=1e-6)
    xs = x.cpu().numpy()
    assert st["converged"]
    # true residual checked with the oracle's operator
    assert np.linalg.norm(b - P.apply(xs)) / np.linalg.norm(b) <= 1e-6 * (1 + 1e-6)
    assert _rel(xs, u_ref) < 1e-5


def test_full_size_2d_layered_operator_and_identities(native):
    """1024^2 + 32-cell PML layered medium at full size: the operator against the
    oracle everywhere; psi_1 / exp consistency M psi_1(M) v = exp(M) v - v
    (Def. psi) through the GPU path in complex128."""
    grid, c, p = I.config_2d_layered()
    P, G = _pair(native, grid, c, p, exp_tol=1e-10)
    x = I.random_complex(grid.n_total, 6)
    xd = _cuda(x)
    ref = P.apply(x, shifted=True)
    got = G.apply_operator(xd, shifted=True).cpu().numpy()
    assert _rel(got, ref) < 1e-13
    e = G.apply_phi(0, xd)[0]
    s = G.apply_phi(1, xd)[0]
    Ms = (1j * p.t) * G.apply_operator(s, shifted=True)
    lhs = Ms.cpu().numpy()
    rhs = (e - xd).cpu().numpy()
    assert _rel(lhs, rhs) < 1e-8
