"""Pins for the oracle's matrix-function actions exp(M)v and psi_1(M)v,
M = i t A_s (Def. psi; Sec. 3.1)."""
import cmath
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2506_03617_gb300 import inputs as I


def _sine_mode(shape_xyz, modes):
    u = np.ones(1)
    for n, a in zip(shape_xyz, modes):
        u = np.multiply.outer(np.sin(math.pi * a * (np.arange(n) + 1) / (n + 1)), u)
    return u.ravel().astype(complex)


@pytest.mark.parametrize("modes", [(1, 2), (5, 3), (8, 7)])
def test_sine_mode_scalar_closed_form(modes):
    """On an eigenvector the actions reduce to the scalar functions
    exp(i t lam) and psi_1(z) = (e^z - 1)/z (Def. psi)."""
    ni, omega, s, t = (9, 8), 5.0, 0.3, 40.0 / 81
    P = oracle.Problem(2, ni, 0, np.ones(72), omega, s, t)
    h = 1.0 / 9
    lam = omega ** 2 * (1 + 1j * s)
    for n, a in zip(ni, modes):
        lam -= 4 / h ** 2 * math.sin(math.pi * a / (2 * (n + 1))) ** 2
    u = _sine_mode(ni, modes)
    z = 1j * t * lam
    assert np.allclose(P.expv(u), cmath.exp(z) * u, atol=1e-12)
    assert np.allclose(P.psi1v(u), (cmath.exp(z) - 1) / z * u, atol=1e-12)


@pytest.mark.parametrize("dim,ni,npml,medium", [(2, (10, 8), 3, "grf"), (3, (4, 4, 3), 2, "one")])
def test_dense_expm_with_pml(dim, ni, npml, medium):
    """Against scipy's dense expm of the assembled matrix M = i t A_s, with psi_1
    read off the augmented matrix [[M, v], [0, 0]] (exp of it gives psi_1(M)v
    in the last column)."""
    g = I.Grid(dim, ni, npml)
    c = I.homogeneous(g) if medium == "one" else I.layered_grf(g, seed=11, corr_cells=2.0)
    p = I.paper_params(g, c, ppw=10.0)
    P = oracle.Problem.from_grid(g, c, p)
    M = 1j * p.t * P.dense(shifted=True)
    n = P.n_total
    v = I.random_complex(n, 2)
    ref_exp = sla.expm(M) @ v
    B = np.zeros((n + 1, n + 1), complex)
    B[:n, :n] = M
    B[:n, n] = v
    ref_psi = sla.expm(B)[:n, n]
    e1 = np.linalg.norm(P.expv(v) - ref_exp) / np.linalg.norm(ref_exp)
    e2 = np.linalg.norm(P.psi1v(v) - ref_psi) / np.linalg.norm(ref_psi)
    assert e1 < 1e-12 and e2 < 1e-12, (e1, e2)


def test_semigroup_and_psi1_identity():
    """exp(2M) = exp(M) exp(M) and M psi_1(M) v = exp(M) v - v."""
    g = I.Grid(2, (12, 12), 4)
    c = I.layered_grf(g, seed=5, corr_cells=3.0)
    p = I.paper_params(g, c, ppw=10.0)
    P1 = oracle.Problem.from_grid(g, c, p)
    P2 = oracle.Problem(2, g.ni, g.npml, c, p.omega, p.shift, 2 * p.t)
    v = I.random_complex(g.n_total, 4)
    e1 = P1.expv(v)
    lhs = P2.expv(v)
    rhs = P1.expv(e1)
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(lhs) < 1e-12
    psi = P1.psi1v(v)
    Mpsi = 1j * p.t * P1.apply(psi, shifted=True)
    assert np.linalg.norm(Mpsi - (e1 - v)) / np.linalg.norm(e1 - v) < 1e-12


def test_unshifted_variant_differs_by_shift_factor_on_homogeneous_medium():
    """With c = 1, A_s = A + i omega^2 s I commutes with A, so
    exp(i t A_s) v = exp(-t omega^2 s) exp(i t A) v."""
    g = I.Grid(2, (10, 10), 3)
    c = I.homogeneous(g)
    p = I.paper_params(g, c, ppw=10.0)
    P = oracle.Problem.from_grid(g, c, p)
    v = I.random_complex(g.n_total, 8)
    a = P.phi(0, v, shifted=True)[0]
    b = P.phi(0, v, shifted=False)[0] * math.exp(-p.t * p.omega ** 2 * p.shift)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-12
