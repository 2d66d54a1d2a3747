"""Pins for the oracle's psi_2 action and for the preconditioner built on the
second inverse formula of Sec. 3.1, A^{-1} = -i t (I - psi_1(i t A))^{-1} psi_2(i t A)
(Def. psi: psi_2(z) = (psi_1(z) - 1)/z = (e^z - 1 - z)/z^2)."""
import cmath
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2506_03617_gb300 import inputs as I


def _sine_mode(ni, modes):
    u = np.ones(1)
    for n, a in zip(ni, modes):
        u = np.multiply.outer(np.sin(math.pi * a * (np.arange(n) + 1) / (n + 1)), u)
    return u.ravel().astype(complex)


@pytest.mark.parametrize("modes", [(1, 1), (4, 6), (8, 8)])
def test_psi2_on_sine_modes_is_the_scalar_function(modes):
    """No PML, c = 1: a sine mode is an eigenvector of A_s with the closed-form
    eigenvalue, so psi_2(i t A_s) u = (e^z - 1 - z)/z^2 u with z = i t lambda."""
    ni, omega, s, t = (9, 8), 5.0, 0.3, 40.0 / 81
    P = oracle.Problem(2, ni, 0, np.ones(72), omega, s, t)
    h = 1.0 / 9
    lam = omega ** 2 * (1 + 1j * s)
    for n, a in zip(ni, modes):
        lam -= 4 / h ** 2 * math.sin(math.pi * a / (2 * (n + 1))) ** 2
    z = 1j * t * lam
    u = _sine_mode(ni, modes)
    want = (cmath.exp(z) - 1 - z) / z ** 2
    got, _ = P.phi(2, u)
    assert np.allclose(got, want * u, atol=1e-12, rtol=0)


@pytest.mark.parametrize("dim,ni,npml", [(2, (9, 7), 3), (3, (3, 4, 3), 2)])
def test_psi2_against_dense_expm_of_the_augmented_matrix(dim, ni, npml):
    """exp([[M, v, 0], [0, 0, 1], [0, 0, 0]]) has psi_2(M) v in its last column
    (the block-triangular exponential integrates exp((1 - s) M) v s over [0, 1])."""
    g = I.Grid(dim, ni, npml)
    c = I.layered_grf(g, seed=17, corr_cells=2.0)
    p = I.paper_params(g, c, ppw=10.0)
    P = oracle.Problem.from_grid(g, c, p)
    n = P.n_total
    M = 1j * p.t * P.dense(shifted=True)
    v = I.random_complex(n, 8)
    B = np.zeros((n + 2, n + 2), complex)
    B[:n, :n] = M
    B[:n, n] = v
    B[n, n + 1] = 1.0
    ref = sla.expm(B)[:n, n + 1]
    got, _ = P.phi(2, v)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_psi2_recurrence_of_def_psi():
    """M psi_2(M) v = psi_1(M) v - v (Def. psi with l = 1)."""
    g = I.Grid(2, (12, 10), 4)
    c = I.layered_grf(g, seed=19, corr_cells=3.0)
    p = I.paper_params(g, c, ppw=10.0)
    P = oracle.Problem.from_grid(g, c, p)
    v = I.random_complex(g.n_total, 9)
    p2, _ = P.phi(2, v)
    lhs = 1j * p.t * P.apply(p2, shifted=True)
    rhs = P.psi1v(v) - v
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-12


def test_second_formula_converged_apply_is_the_scaled_inverse():
    """Solving (I - psi_1(i t A_s)) w = psi_2(i t A_s) r exactly gives
    w = (i/t) A_s^{-1} r, as for Algorithm 1."""
    g = I.Grid(2, (12, 12), 4)
    c = I.layered_grf(g, seed=21, corr_cells=3.0)
    p = I.paper_params(g, c, ppw=10.0)
    P = oracle.Problem.from_grid(g, c, p)
    r = I.random_complex(g.n_total, 10)
    w, it, _ = P.matexpre(r, fprtol=1e-13, restart=400, maxit=400, variant=1)
    ref = (1j / p.t) * np.linalg.solve(P.dense(shifted=True), r)
    assert np.linalg.norm(w - ref) / np.linalg.norm(ref) < 1e-9
    assert it < 400


def test_second_formula_inner_residual_meets_fprtol():
    g = I.Grid(2, (10, 10), 3)
    c = I.layered_grf(g, seed=23, corr_cells=3.0)
    p = I.paper_params(g, c, ppw=10.0)
    P = oracle.Problem.from_grid(g, c, p)
    r = I.random_complex(g.n_total, 12)
    w, it, _ = P.matexpre(r, fprtol=0.08, variant=1)
    rt, _ = P.phi(2, r)
    res = rt - (w - P.psi1v(w))
    assert np.linalg.norm(res) <= 0.08 * np.linalg.norm(rt) * (1 + 1e-9)
    assert it >= 1


def test_fgmres_with_the_second_formula_reaches_the_direct_solution():
    g = I.Grid(2, (24, 24), 6)
    c = I.layered_grf(g, seed=25, corr_cells=3.0)
    p = I.paper_params(g, c, ppw=10.0)
    P = oracle.Problem.from_grid(g, c, p)
    b = I.rhs_from_source(I.gaussian_source(g)).ravel()
    u, info = P.fgmres(b, rtol=1e-8, variant=1)
    assert info["converged"] and info["true_relres"] <= 1e-8
    ref = np.linalg.solve(P.dense(), b)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-6
