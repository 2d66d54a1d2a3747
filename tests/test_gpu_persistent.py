"""GPU parity of the persistent exp-action kernel (one cooperative launch per
action, tiles held in shared memory, K-wide halo exchange through L2 between
passes) against the per-pass sweeps and the fp64 oracle, element-wise over the
interior and the PML cells.  Every configuration must run on at least one grid
for each storage type and action (checked at the end of the module)."""
import numpy as np
import pytest

import oracle
from paper_2506_03617_gb300 import inputs as I

from _parity import TOL_LOW, check

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


RAN = {}     # (action, prec) -> configurations that ran on some grid


@pytest.mark.parametrize("grid", [I.Grid(2, (290, 157), 6), I.Grid(2, (64, 64), 10),
                                  I.Grid(2, (3, 40), 4)])
@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_persistent_matches_per_pass_and_oracle(native, grid, prec):
    c = I.layered_grf(grid, seed=41, corr_cells=3.0)
    p = I.paper_params(grid, c, ppw=10.0)
    P = oracle.Problem.from_grid(grid, c, p)
    x = I.random_complex(grid.n_total, 11)
    xd = torch.from_numpy(x).cuda()
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec=prec, exp_tol=1e-6, fuse_k=1, persist_cfg=-2)
    base = G.apply_phi(0, xd)[0].cpu().numpy()
    ref = P.phi(0, x)[0]
    ran = RAN.setdefault(("exp", prec), set())
    for cfg in range(native.load().mxp_num_persist_configs()):
        G.set_params(fuse_k=0, persist_cfg=cfg)
        if G.persist_config()[0] != cfg:
            continue                          # the grid does not fit this configuration
        ran.add(cfg)
        got = G.apply_phi(0, xd)[0].cpu().numpy()
        check(got, ref, grid, TOL_LOW[prec], what=f"persist cfg {cfg} exp {prec}")
        if prec == "c64":
            assert _rel(got, base) < 5e-5, (cfg, _rel(got, base))


def test_persistent_on_the_1088_workload_and_solve(native):
    grid, c, p = I.config_2d_layered()
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec="c64", exp_tol=1e-6, persist_cfg=0)
    assert G.persist_config()[0] == 0
    RAN.setdefault(("exp", "c64"), set()).add(0)
    x = torch.from_numpy(I.random_complex(grid.n_total, 12)).cuda()
    e = G.apply_phi(0, x)[0]
    G.set_params(persist_cfg=-2, fuse_k=1)
    e_ref = G.apply_phi(0, x)[0]
    assert _rel(e.cpu().numpy(), e_ref.cpu().numpy()) < 5e-5
    # automatic choice, then a full solve: true residual checked by the oracle's operator
    G.set_params(persist_cfg=-1, fuse_k=0)
    b = I.rhs_from_source(I.gaussian_source(grid)).ravel()
    xs, st = G.solve(torch.from_numpy(b).cuda(), rtol=1e-6)
    assert st["converged"]
    P = oracle.Problem.from_grid(grid, c, p)
    xs = xs.cpu().numpy()
    assert np.linalg.norm(b - P.apply(xs)) / np.linalg.norm(b) <= 1.000001e-6


def test_persistent_refuses_grids_that_do_not_fit(native):
    grid = I.Grid(2, (3000, 3000), 8)
    c = I.homogeneous(grid)
    p = I.paper_params(grid, c, ppw=10.0)
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec="c64", exp_tol=1e-6, persist_cfg=0)
    assert G.persist_config()[0] == -1


@pytest.mark.parametrize("grid", [I.Grid(2, (290, 157), 6), I.Grid(2, (64, 64), 10)])
@pytest.mark.parametrize("prec", ["c64", "bf16s"])
def test_persistent_psi1_matches_per_pass_and_oracle(native, grid, prec):
    """psi_1 on the persistent kernel (first sub-step per point, the rest in one
    launch adding c_j w after every sub-step) against the per-pass sweeps and the
    oracle, for every configuration that fits; also the fixed-point operator
    x - psi_1 x of the second inverse formula."""
    c = I.layered_grf(grid, seed=43, corr_cells=3.0)
    p = I.paper_params(grid, c, ppw=10.0)
    P = oracle.Problem.from_grid(grid, c, p)
    x = I.random_complex(grid.n_total, 21)
    xd = torch.from_numpy(x).cuda()
    G = native.Problem.from_grid(grid, c, p)
    G.set_params(prec=prec, exp_tol=1e-6, fuse_k=1, persist_cfg=-2)
    base = G.apply_phi(1, xd)[0].cpu().numpy()
    ref = P.phi(1, x)[0]
    ran = RAN.setdefault(("psi1", prec), set())
    for cfg in range(native.load().mxp_num_persist_configs()):
        G.set_params(fuse_k=0, persist_cfg=cfg)
        if G.persist_config()[0] != cfg:
            continue
        ran.add(cfg)
        got = G.apply_phi(1, xd)[0].cpu().numpy()
        check(got, ref, grid, TOL_LOW[prec], what=f"persist cfg {cfg} psi1 {prec}")
        if prec == "c64":
            assert _rel(got, base) < 5e-5, (cfg, _rel(got, base))
    # the second inverse formula's apply runs psi_1 actions on this path
    G.set_params(precond=2, inner_fixed=3, exp_tol=1e-6)
    r = I.random_complex(grid.n_total, 22)
    w_ref, it, _ = P.matexpre(r, fixed=3, variant=1)
    w, st = G.apply_matexpre(torch.from_numpy(r).cuda())
    assert st["inner_iters"] == 3
    check(w.cpu().numpy(), w_ref, grid, TOL_LOW[prec], what=f"psi2-variant apply {prec}")


def test_every_configuration_ran(native):
    """No configuration was skipped everywhere: each one, for both storage types
    and both actions, met the oracle on at least one grid above."""
    every = set(range(native.load().mxp_num_persist_configs()))
    for key in [("exp", "c64"), ("exp", "bf16s"), ("psi1", "c64"), ("psi1", "bf16s")]:
        assert RAN.get(key, set()) == every, (key, sorted(RAN.get(key, set())))

