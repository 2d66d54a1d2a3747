"""Failure detection without a GPU fault: a bounded device-side wait that runs
out returns MXP_ETIMEOUT and the problem stays usable; invalid inputs are
rejected on the host before any device work; a NaN right-hand side is
reported as MXP_ENAN."""
import numpy as np
import pytest

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


def _small(native):
    g = I.Grid(2, (40, 36), 6)
    c = I.homogeneous(g)
    p = I.paper_params(g, c, ppw=10.0)
    return g, native.Problem.from_grid(g, c, p)


def test_barrier_wait_times_out_and_the_problem_stays_usable(native):
    g, G = _small(native)
    s = native.load().mxp_selftest_barrier_timeout(G._h)
    assert s == 7, native.load().mxp_last_error()          # MXP_ETIMEOUT
    x = torch.from_numpy(I.random_complex(g.n_total, 1)).cuda()
    y = G.apply_operator(x)
    assert torch.isfinite(torch.view_as_real(y)).all()
    b = torch.from_numpy(I.rhs_from_source(I.gaussian_source(g)).ravel()).cuda()
    _, st = G.solve(b, rtol=1e-6)
    assert st["converged"]


def test_nan_rhs_is_reported(native):
    g, G = _small(native)
    b = torch.full((g.n_total,), float("nan"), dtype=torch.complex128, device="cuda")
    with pytest.raises(native.MxpError) as e:
        G.solve(b, rtol=1e-6)
    assert e.value.status == 6                                # MXP_ENAN


def test_invalid_parameters_are_rejected(native):
    g, G = _small(native)
    for bad in (dict(omega=-1.0), dict(fprtol=1.5), dict(t=0.0), dict(inner_restart=0),
                dict(tile_cfg=999), dict(persist_cfg=99)):
        with pytest.raises(native.MxpError) as e:
            G.set_params(**bad)
        assert e.value.status == 1
    with pytest.raises(native.MxpError):
        native.Problem(2, (4, 4), 1, -np.ones(36))


def test_timeout_survives_a_later_persistent_launch(native):
    """The error word of a timed-out wait is kept by the next persistent launch
    (which used to clear it before starting) until the host reads it; the
    problem's next action is then correct again."""
    g = I.Grid(2, (120, 100), 8)
    c = I.layered_grf(g, seed=I.SEED_BASE + 17, corr_cells=4.0)
    p = I.paper_params(g, c, ppw=10.0)
    G = native.Problem.from_grid(g, c, p)
    G.set_params(prec="c64", exp_tol=1e-6, persist_cfg=6)
    assert G.persist_config()[0] == 6
    s = native.load().mxp_selftest_barrier_timeout(G._h)
    assert s == 7, native.load().mxp_last_error()          # MXP_ETIMEOUT
    x = torch.from_numpy(I.random_complex(g.n_total, 3)).cuda()
    got = G.apply_phi(0, x)[0].cpu().numpy()
    G.set_params(persist_cfg=-2, fuse_k=1)
    ref = G.apply_phi(0, x)[0].cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 5e-5
