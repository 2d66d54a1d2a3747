"""GPU parity of the fused 2D Taylor-Horner sweeps (complex64 and
bfloat16-storage): every tile configuration against the unfused kernel and
against the fp64 oracle, on grids that span several tiles with ragged tails,
grids smaller than one tile, and PML-heavy grids."""
import numpy as np
import pytest

import oracle
from paper_2506_03617_gb300 import inputs as I

from _parity import TOL_LOW, TOL_POINTWISE, check

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


GRIDS = [I.Grid(2, (290, 157), 6), I.Grid(2, (20, 12), 3), I.Grid(2, (1, 40), 4),
         I.Grid(2, (130, 30), 24)]


@pytest.mark.parametrize("gi", range(len(GRIDS)))
@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_every_tile_config_matches_unfused_and_oracle(native, gi, prec):
    grid = GRIDS[gi]
    c = I.layered_grf(grid, seed=31 + gi, corr_cells=3.0)
    p = I.paper_params(grid, c, ppw=10.0)
    P = oracle.Problem.from_grid(grid, c, p)
    x = I.random_complex(grid.n_total, 7)
    xd = torch.from_numpy(x).cuda()
    G = native.Problem.from_grid(grid, c, p)
    bound = TOL_LOW[prec]
    for which in (0, 1):
        ref = P.phi(which, x)[0]
        G.set_params(prec=prec, exp_tol=1e-6, fuse_k=1, tile_cfg=-1)
        assert G.tile_config()[0] == -1
        base = G.apply_phi(which, xd)[0].cpu().numpy()
        check(base, ref, grid, TOL_POINTWISE[prec], what=f"unfused phi{which} {prec}")
        for cfg in range(native.load().mxp_num_tile_configs()):
            G.set_params(fuse_k=0, tile_cfg=cfg)
            assert G.tile_config()[0] == cfg
            got = G.apply_phi(which, xd)[0].cpu().numpy()
            check(got, ref, grid, bound, what=f"fused2d cfg {cfg} phi{which} {prec}")
            if prec == "c64":
                # same arithmetic up to float rounding order (plan may add steps for K | m)
                assert _rel(got, base) < 5e-5, (cfg, which, _rel(got, base))


def test_autotuner_picks_a_fused_config_on_the_2d_workload(native):
    grid, c, p = I.config_2d_layered()
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec="c64", exp_tol=1e-6)
    cfg, k = G.tile_config()
    assert cfg >= -1
    x = torch.from_numpy(I.random_complex(grid.n_total, 9)).cuda()
    e, _ = G.apply_phi(0, x)
    s, _ = G.apply_phi(1, x)
    # Def. psi: M psi_1(M) x = exp(M) x - x, checked in fp64 through the operator
    lhs = ((1j * p.t) * G.apply_operator(s, shifted=True)).cpu().numpy()
    rhs = (e - x).cpu().numpy()
    assert _rel(lhs, rhs) < 5e-4
