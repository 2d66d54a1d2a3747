"""Pins for the oracle's Algorithm 1 (MatExPre preconditioning step) and the
outer FGMRES solve."""
import math

import numpy as np
import pytest
import scipy.special as ssp
import scipy.sparse.linalg as spla

import oracle
from paper_2506_03617_gb300 import inputs as I
from _sparse import probe_sparse


def _small(seed=7, ni=(14, 12), npml=4, medium="grf"):
    g = I.Grid(2, ni, npml)
    c = I.homogeneous(g) if medium == "one" else I.layered_grf(g, seed=seed, corr_cells=3.0)
    p = I.paper_params(g, c, ppw=10.0)
    return g, c, p, oracle.Problem.from_grid(g, c, p)


def test_converged_apply_equals_scaled_inverse():
    """Eq. magic-inverse / Eq. inverse-1 with the constant -i t dropped: solving
    (I - exp(i t A_s)) w = psi_1(i t A_s) r exactly gives w = (i/t) A_s^{-1} r."""
    g, c, p, P = _small()
    r = I.random_complex(g.n_total, 3)
    w, it, _ = P.matexpre(r, fprtol=1e-13, restart=400, maxit=400)
    As = P.dense(shifted=True)
    ref = (1j / p.t) * np.linalg.solve(As, r)
    assert np.linalg.norm(w - ref) / np.linalg.norm(ref) < 1e-9
    assert it < 400


def test_inner_residual_meets_fprtol():
    """The returned w satisfies ||r~ - (I - e^{itA_s}) w|| <= fprtol ||r~||, with
    r~ = psi_1(i t A_s) r (Algorithm 1)."""
    g, c, p, P = _small(seed=9)
    r = I.random_complex(g.n_total, 5)
    w, it, _ = P.matexpre(r, fprtol=0.08)
    rt = P.psi1v(r)
    res = rt - (w - P.expv(w))
    assert np.linalg.norm(res) <= 0.08 * np.linalg.norm(rt) * (1 + 1e-9)
    assert it >= 1


def test_fixed_trip_mode_is_linear_in_r():
    """With a fixed number of inner iterations the apply is a fixed polynomial in
    the Krylov space of r~, hence homogeneous: P(a r) = a P(r)."""
    g, c, p, P = _small(seed=13, ni=(10, 10), npml=3)
    r = I.random_complex(g.n_total, 6)
    w1, it1, _ = P.matexpre(r, fixed=4)
    w2, it2, _ = P.matexpre((2 - 3j) * r, fixed=4)
    assert it1 == it2 == 4
    assert np.linalg.norm(w2 - (2 - 3j) * w1) / np.linalg.norm(w2) < 1e-12


def test_fgmres_converges_to_direct_solution():
    """Outer FGMRES with Algorithm 1 as right preconditioner reaches the direct
    solution of A u = b (unshifted A)."""
    g, c, p, P = _small(seed=17, ni=(20, 18), npml=5)
    b = I.rhs_from_source(I.gaussian_source(g)).ravel()
    u, info = P.fgmres(b, rtol=1e-10, restart=30, maxit=60)
    assert info["converged"]
    ref = np.linalg.solve(P.dense(), b)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-8
    assert info["true_relres"] <= 1e-10
    h = info["res_hist"]
    assert np.all(np.diff(h[: min(len(h), 30)]) <= 1e-12 * h[0])   # GMRES minimal residual


def test_point_source_matches_outgoing_hankel_far_field():
    """With e^{-i w t} time dependence (Sec. 2) the outgoing 2D free-space
    solution of Lap u + k^2 u = -f is (i/4) H_0^(1)(k r) convolved with f; for
    the normalised Gaussian f of width sigma it is ~ (i/4) H_0^(1)(k r)
    exp(-k^2 sigma^2 / 2) away from the source.  The PML must absorb (no
    reflection) for the comparison to hold."""
    N, npml, ppw = 96, 24, 32.0
    g = I.Grid(2, (N, N), npml)
    c = I.homogeneous(g)
    h = g.h
    k = 2 * math.pi / (ppw * h)
    P = oracle.Problem(2, g.ni, npml, c, k, 0.0, 1.0)
    f = I.gaussian_source(g, sigma_cells=1.0).ravel()
    A = probe_sparse(lambda v: P.apply(v), g.n)
    u = spla.spsolve(A.tocsc(), -f)
    # note A u = -f means Lap u + k^2 u = -f
    x = g.node_coords(0)
    X, Y = np.meshgrid(x, x)                    # [y][x]
    r = np.hypot(X - 0.5, Y - 0.5).ravel()
    ring = (r > 0.15) & (r < 0.42)
    ref = 0.25j * ssp.hankel1(0, k * r[ring]) * math.exp(-(k * h) ** 2 / 2)
    err = np.linalg.norm(u[ring] - ref) / np.linalg.norm(ref)
    assert err < 0.08, err
