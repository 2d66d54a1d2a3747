"""GPU parity of the fused 3D sweeps (z-marching temporal blocking, complex64
and bfloat16 storage): every configuration against the unfused kernel and the
fp64 oracle on ragged 3D grids, and the full-size 288^3 exp action against the
unfused kernel."""
import numpy as np
import pytest

import oracle
from paper_2506_03617_gb300 import inputs as I

from _parity import TOL_LOW, TOL_POINTWISE, check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N3 = 4


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03617_gb300 import native as N
    N.load()
    return N


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("grid", [I.Grid(3, (41, 29, 17), 3), I.Grid(3, (20, 70, 9), 4),
                                  I.Grid(3, (6, 6, 40), 2)])
@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_fused3d_matches_unfused_and_oracle(native, grid, prec):
    c = I.layered_grf(grid, seed=51, corr_cells=3.0)
    p = I.paper_params(grid, c, ppw=10.0)
    P = oracle.Problem.from_grid(grid, c, p)
    x = I.random_complex(grid.n_total, 13)
    xd = torch.from_numpy(x).cuda()
    ref = P.phi(0, x)[0]
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec=prec, exp_tol=1e-6, fuse_k=1, tile_cfg=-1)
    assert G.tile_config()[0] == -1
    base = G.apply_phi(0, xd)[0].cpu().numpy()
    bound = TOL_LOW[prec]
    check(base, ref, grid, TOL_POINTWISE[prec], what=f"3d unfused exp {prec}")
    for cfg in range(N3):
        G.set_params(fuse_k=0, tile_cfg=cfg)
        assert G.tile_config()[0] == cfg
        got = G.apply_phi(0, xd)[0].cpu().numpy()
        check(got, ref, grid, bound, what=f"fused3d cfg {cfg} exp {prec}")
        if prec == "c64":
            assert _rel(got, base) < 5e-5, (cfg, _rel(got, base))
    # psi_1 keeps working on the 3D path (unfused sweeps)
    s = G.apply_phi(1, xd)[0].cpu().numpy()
    check(s, P.phi(1, x)[0], grid, TOL_POINTWISE[prec], what=f"3d psi1 {prec}")


def test_full_size_288_exp_action_fused_vs_unfused(native):
    grid, c, p = I.config_3d_homogeneous()
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec="c64", exp_tol=1e-6, fuse_k=1)
    x = torch.from_numpy(I.random_complex(grid.n_total, 14)).cuda()
    base = G.apply_phi(0, x)[0]
    G.set_params(fuse_k=0, tile_cfg=-1)
    got = G.apply_phi(0, x)[0]
    assert _rel(got.cpu().numpy(), base.cpu().numpy()) < 5e-5


@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_low_precision_3d_solve_reaches_tolerance(native, prec):
    """FGMRES with complex64 / bf16-storage 3D sweeps (z-marching kernel) on a
    ragged lens grid reaches the 1e-6 true residual of the fp64 operator."""
    grid = I.Grid(3, (33, 27, 21), 4)
    c = I.lens(grid)
    p = I.paper_params(grid, c, ppw=10.0)
    P = oracle.Problem.from_grid(grid, c, p)
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec=prec, exp_tol=1e-6)
    b = I.rhs_from_source(I.gaussian_source(grid)).ravel()
    x, st = G.solve(torch.from_numpy(b).cuda(), rtol=1e-6, maxit=300)
    assert st["converged"]
    assert np.linalg.norm(b - P.apply(x.cpu().numpy())) / np.linalg.norm(b) <= 1.000001e-6
