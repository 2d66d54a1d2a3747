"""GPU parity: the CUDA path (through the C ABI) against the fp64 oracle.

Every comparison is element-wise (the largest error over the interior cells
and over the PML cells, relative to max|ref|) with the l2 norm alongside
(tests/_parity.py).  Bounds: 1e-13 for the operator, 1e-10 per exp / psi_1 /
MatExPre application in complex128 with the inner iteration count fixed
(exp_tol 1e-12), 1e-8 on the final solution at the same outer count (config
c1: 128^2 + 16 PML at the paper's parameters, FGMRES(30)); the complex64 and
bfloat16-storage errors are bounded by TOL_C64 / TOL_BF16S, including the
kernel the benchmark times on the full 1088^2 workload."""
import numpy as np
import pytest

import oracle
from paper_2506_03617_gb300 import inputs as I

from _parity import TOL_C128, TOL_LOW, TOL_OP, TOL_SOLUTION, check, errors

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
    check(got, ref, grid, TOL_OP, what=f"operator {name} shifted={shifted}")


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
    check(got.cpu().numpy(), ref, grid, TOL_C128, what=f"phi{which} c128 {name}")


def test_matexpre_fixed_trip_parity_c128(native):
    grid = I.Grid(2, (40, 36), 6)
    c = _medium(grid, "grf")
    p = I.paper_params(grid, c, ppw=10.0)
    P, G = _pair(native, grid, c, p, exp_tol=1e-12, inner_fixed=3)
    r = I.random_complex(grid.n_total, 3)
    ref, it, _ = P.matexpre(r, fixed=3)
    got, st = G.apply_matexpre(_cuda(r))
    assert st["inner_iters"] == it == 3
    check(got.cpu().numpy(), ref, grid, TOL_C128, what="matexpre fixed 3 c128")


def test_matexpre_tolerance_mode_matches_iterations(native):
    grid = I.Grid(2, (40, 36), 6)
    c = _medium(grid, "grf")
    p = I.paper_params(grid, c, ppw=10.0)
    P, G = _pair(native, grid, c, p, exp_tol=1e-12)
    r = I.random_complex(grid.n_total, 4)
    ref, it, _ = P.matexpre(r, fprtol=0.08)
    got, st = G.apply_matexpre(_cuda(r))
    assert st["inner_iters"] == it
    check(got.cpu().numpy(), ref, grid, TOL_C128, what="matexpre tolerance mode c128")


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
    check(x.cpu().numpy(), u_ref, grid, TOL_SOLUTION, what="solve 64^2+10 c128")


def test_solve_parity_config_c1(native):
    """Config c1 as specified: 128^2 interior + 16-cell PML, c = 1, ppw 10, the
    paper's s, t, C_pml and fprtol, Gaussian source at the centre, FGMRES(30) to
    a relative residual of 1e-6 with complex128 actions (exp_tol 1e-12).  The
    GPU solve takes the oracle's outer and inner iteration counts and its
    solution agrees element-wise within 1e-8."""
    grid, c, p = I.config_2d_homogeneous()
    P, G = _pair(native, grid, c, p, exp_tol=1e-12)
    b = I.rhs_from_source(I.gaussian_source(grid)).ravel()
    u_ref, info = P.fgmres(b, rtol=1e-6, restart=30)
    x, st = G.solve(_cuda(b), rtol=1e-6, restart=30)
    assert st["converged"] and info["converged"]
    assert st["outer_iters"] == info["outer_iters"]
    assert st["inner_iters_total"] == sum(info["inner"])
    check(x.cpu().numpy(), u_ref, grid, TOL_SOLUTION, what="solve c1 c128")


@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_low_precision_phi_error_bounded(native, prec):
    grid = I.Grid(2, (40, 36), 6)
    c = _medium(grid, "grf")
    p = I.paper_params(grid, c, ppw=10.0)
    P, G = _pair(native, grid, c, p, prec=prec, exp_tol=1e-6)
    x = I.random_complex(grid.n_total, 5)
    for which in (0, 1):
        ref = P.phi(which, x)[0]
        got = G.apply_phi(which, _cuda(x))[0].cpu().numpy()
        check(got, ref, grid, TOL_LOW[prec], what=f"phi{which} {prec} 40x36+6")


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
    check(xs, u_ref, grid, 1e-5, what=f"solve 64^2+10 {prec}")


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
    check(got, ref, grid, TOL_OP, what="operator 1088^2")
    e = G.apply_phi(0, xd)[0]
    s = G.apply_phi(1, xd)[0]
    Ms = (1j * p.t) * G.apply_operator(s, shifted=True)
    check(Ms.cpu().numpy(), (e - xd).cpu().numpy(), grid, 1e-8, what="Def. psi identity 1088^2 c128")


def test_benched_kernel_on_the_full_1088_workload_against_the_oracle(native):
    """The kernel the benchmark times, in the launch configuration it times: the
    autotuner's choice for complex64 on the full 1024^2 + 32 layered workload
    (the persistent exp-action kernel) with the benchmark's Taylor plan.  Checked element-wise against the fp64
    oracle on the full grid: the exp action at the workload's t, and the exp and
    psi_1 actions at t/16 with the same configuration forced."""
    grid, c, p = I.config_2d_layered()
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec="c64", exp_tol=1e-3, theta_max=6.0)       # the benchmark's plan
    cfg, ntiles = G.persist_config()
    assert cfg >= 0, "the autotuner no longer picks the persistent kernel on this workload"
    x = I.random_complex(grid.n_total, 31)
    xd = _cuda(x)
    P = oracle.Problem.from_grid(grid, c, p)
    got = G.apply_phi(0, xd)[0].cpu().numpy()
    check(got, P.phi(0, x)[0], grid, TOL_LOW["c64"], what=f"benched kernel cfg {cfg} exp full t")
    # the same configuration at t/16: fewer sub-steps, same tiles
    p16 = I.Params(omega=p.omega, shift=p.shift, t=p.t / 16, cpml=p.cpml, fprtol=p.fprtol)
    G.set_params(t=p16.t, persist_cfg=cfg)
    assert G.persist_config() == (cfg, ntiles)
    P16 = oracle.Problem.from_grid(grid, c, p16)
    for which in (0, 1):
        got = G.apply_phi(which, xd)[0].cpu().numpy()
        check(got, P16.phi(which, x)[0], grid, TOL_LOW["c64"], what=f"benched kernel cfg {cfg} phi{which} t/16")


@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_pml_and_interior_errors_are_reported_separately(native, prec):
    """The element-wise check sees a PML-heavy grid's PML cells on their own: a
    grid whose PML holds most of the unknowns keeps both maxima in bound."""
    grid = I.Grid(2, (30, 26), 24)
    c = _medium(grid, "grf")
    p = I.paper_params(grid, c, ppw=10.0)
    P, G = _pair(native, grid, c, p, prec=prec, exp_tol=1e-6)
    x = I.random_complex(grid.n_total, 8)
    got = G.apply_phi(0, _cuda(x))[0].cpu().numpy()
    e = check(got, P.phi(0, x)[0], grid, TOL_LOW[prec], what=f"phi0 {prec} PML-heavy")
    assert e["max_pml"] > 0 and e["max_int"] > 0
    assert errors(got, got, grid)["max_pml"] == 0.0


@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_performance_plan_accuracy(native, prec):
    """The benchmark's Taylor plan (exp_tol 1e-3, theta_max 6: about a quarter
    fewer sweeps than exp_tol 1e-6, theta_max 4) keeps the low-precision
    actions within the same bounds of the fp64 oracle, since below float
    rounding a tighter truncation buys nothing; the solve still reaches the
    1e-6 true residual."""
    grid = I.Grid(2, (96, 80), 10)
    c = _medium(grid, "grf")
    p = I.paper_params(grid, c, ppw=8.0)
    P, G = _pair(native, grid, c, p, prec=prec, exp_tol=1e-3, theta_max=6.0)
    x = I.random_complex(grid.n_total, 9)
    for which in (0, 1):
        got = G.apply_phi(which, _cuda(x))[0].cpu().numpy()
        check(got, P.phi(which, x)[0], grid, TOL_LOW[prec], what=f"phi{which} {prec} performance plan")
    b = I.rhs_from_source(I.gaussian_source(grid)).ravel()
    xs, st = G.solve(_cuda(b), rtol=1e-6)
    assert st["converged"]
    assert np.linalg.norm(b - P.apply(xs.cpu().numpy())) / np.linalg.norm(b) <= 1.000001e-6
