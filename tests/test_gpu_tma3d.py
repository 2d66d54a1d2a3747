"""GPU parity of the TMA-staged 3D sweep (complex64 and bf16 storage; planes
brought into shared memory by cp.async.bulk.tensor) against the fp64 oracle,
on ragged grids whose x extent is a multiple of 4 (the kernel's condition);
other grids run the register-marching sweep."""
import numpy as np
import pytest

import oracle
from paper_2506_03617_gb300 import inputs as I

from _parity import TOL_POINTWISE, check

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


GRIDS = [I.Grid(3, (38, 29, 17), 3),     # 44 x 35 x 23: two x tiles, ragged y tiles, several z segments
         I.Grid(3, (60, 20, 9), 2),      # 64 x 24 x 13: whole x tiles
         I.Grid(3, (2, 6, 40), 1)]       # 4 x 8 x 42: one narrow tile, long z


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_tma_sweep_actions_match_oracle(native, grid, prec):
    c = I.layered_grf(grid, seed=61, corr_cells=3.0)
    p = I.paper_params(grid, c, ppw=10.0)
    P = oracle.Problem.from_grid(grid, c, p)
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec=prec, exp_tol=1e-6, fuse_k=1)
    assert G.sweep_kernel() == "zmarch_tma_3d"
    x = I.random_complex(grid.n_total, 17)
    xd = torch.from_numpy(x).cuda()
    for which in (0, 1, 2):
        got = G.apply_phi(which, xd)[0].cpu().numpy()
        ref = P.phi(which, x)[0]
        check(got, ref, grid, TOL_POINTWISE[prec], what=f"tma3d phi{which} {prec}")


def test_odd_x_extent_uses_register_marching(native):
    grid = I.Grid(3, (41, 29, 17), 3)       # n0 = 47
    c = I.homogeneous(grid)
    p = I.paper_params(grid, c, ppw=10.0)
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec="c64", exp_tol=1e-6, fuse_k=1)
    assert G.sweep_kernel() == "zmarch_3d"
    G.set_params(prec="c128", exp_tol=1e-12)
    assert G.sweep_kernel() == "pointwise"


def test_tma_solve_reaches_tolerance(native):
    grid = I.Grid(3, (40, 32, 24), 4)
    c = I.lens(grid)
    p = I.paper_params(grid, c, ppw=10.0)
    P = oracle.Problem.from_grid(grid, c, p)
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec="c64", exp_tol=1e-6)
    assert G.sweep_kernel() == "zmarch_tma_3d"
    b = I.rhs_from_source(I.gaussian_source(grid)).ravel()
    x, st = G.solve(torch.from_numpy(b).cuda(), rtol=1e-6, maxit=300)
    assert st["converged"]
    assert np.linalg.norm(b - P.apply(x.cpu().numpy())) / np.linalg.norm(b) <= 1.000001e-6


def test_full_size_288_tma_matches_fused_kernel(native):
    """The 288^3 exp action through the TMA sweep agrees with the z-marching
    fused kernel (an independent implementation) to complex64 rounding."""
    grid, c, p = I.config_3d_homogeneous()
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec="c64", exp_tol=1e-6, fuse_k=1)
    assert G.sweep_kernel() == "zmarch_tma_3d"
    x = torch.from_numpy(I.random_complex(grid.n_total, 19)).cuda()
    a = G.apply_phi(0, x)[0]
    G.set_params(fuse_k=0, tile_cfg=2)
    assert G.sweep_kernel() == "fused_3d"
    b = G.apply_phi(0, x)[0]
    assert float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) < 5e-5
