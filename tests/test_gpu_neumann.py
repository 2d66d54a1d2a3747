"""The truncated Neumann preconditioner P_N (Sec. 3.2) on the GPU: parity with
the oracle's P_N in complex128, and FGMRES preconditioned by P_N (a fixed linear
map) reaching the 1e-6 true residual."""
import numpy as np
import pytest

import oracle
from paper_2506_03617_gb300 import inputs as I

from _parity import TOL_C128, check

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


@pytest.mark.parametrize("nterms", [0, 3])
def test_neumann_parity_c128(native, nterms):
    g = I.Grid(2, (40, 36), 6)
    c = I.layered_grf(g, seed=81, corr_cells=4.0)
    p = I.paper_params(g, c, ppw=10.0)
    P = oracle.Problem.from_grid(g, c, p)
    G = native.Problem.from_grid(g, c, p)
    G.set_params(exp_tol=1e-12, precond=1, neumann_n=nterms)
    r = I.random_complex(g.n_total, 5)
    w, st = G.apply_matexpre(torch.from_numpy(r).cuda())
    assert st["inner_iters"] == nterms
    check(w.cpu().numpy(), P.neumann(r, nterms), g, TOL_C128, what=f"neumann N={nterms} c128")


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_fgmres_with_neumann_preconditioner_converges(native, prec):
    g = I.Grid(2, (64, 64), 10)
    c = I.homogeneous(g)
    p = I.paper_params(g, c, ppw=10.0)
    G = native.Problem.from_grid(g, c, p)
    G.set_params(prec=prec, exp_tol=1e-12 if prec == "c128" else 1e-6, precond=1, neumann_n=6)
    b = I.rhs_from_source(I.gaussian_source(g)).ravel()
    x, st = G.solve(torch.from_numpy(b).cuda(), rtol=1e-6, maxit=400)
    assert st["converged"]
    P = oracle.Problem.from_grid(g, c, p)
    assert np.linalg.norm(b - P.apply(x.cpu().numpy())) / np.linalg.norm(b) <= 1.000001e-6
