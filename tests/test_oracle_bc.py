"""Pins for the oracle's mixed boundary conditions (Sec. 4, Marmousi-II): a
sound-hard face (du/dn = 0) and first-order absorbing faces (du/dn = i k u),
both through ghost points, on grids without PML."""
import math

import numpy as np
import pytest

import oracle
from paper_2506_03617_gb300 import inputs as I


def _cos_sin_mode(n0, n1, a, b):
    """sin in x (zero Dirichlet ghosts at i = -1 and n0) times cos in y with a
    sound-hard face below j = 0 and a zero ghost at j = n1:
    cos(theta (j + 1/2)), theta = pi (b + 1/2) / (n1 + 1/2)."""
    th = math.pi * (b + 0.5) / (n1 + 0.5)
    ux = np.sin(math.pi * a * (np.arange(n0) + 1) / (n0 + 1))
    uy = np.cos(th * (np.arange(n1) + 0.5))
    return np.multiply.outer(uy, ux).ravel().astype(complex), th


@pytest.mark.parametrize("a,b", [(1, 0), (3, 2), (7, 5)])
def test_sound_hard_face_cosine_eigenpairs(a, b):
    n0, n1 = 11, 9
    omega, s, t = 6.0, 0.2, 0.01
    h = 1.0 / n0
    P = oracle.Problem(2, (n0, n1), 0, np.ones(n0 * n1), omega, s, t, h=h,
                       bc=["dirichlet", "dirichlet", "sound_hard", "dirichlet"])
    u, th = _cos_sin_mode(n0, n1, a, b)
    lam = omega ** 2 * (1 + 1j * s) - 4 / h ** 2 * (math.sin(math.pi * a / (2 * (n0 + 1))) ** 2
                                                   + math.sin(th / 2) ** 2)
    assert np.allclose(P.apply(u, shifted=True), lam * u, atol=1e-9 * abs(lam), rtol=0)


def _plane_wave_residual(n, k):
    """Relative residual of the sampled outgoing wave exp(i k x) in the last
    row (absorbing face x+) and in the interior rows, on an n x 1 grid whose y
    faces are sound-hard (so the field may be constant in y)."""
    h = 1.0 / n
    P = oracle.Problem(2, (n, 1), 0, np.ones(n), k, 0.0, 0.01, h=h,
                       bc=["dirichlet", "absorbing", "sound_hard", "sound_hard"])
    x = (np.arange(n) + 0.5) * h
    u = np.exp(1j * k * x)
    r = P.apply(u)
    return abs(r[-1]) / k ** 2, np.max(np.abs(r[1:-1])) / k ** 2


def test_absorbing_face_is_consistent_with_the_outgoing_wave():
    """The ghost relation reproduces exp(i k h) to third order, so the boundary
    row's residual is O(k h) (k^3 h / 12 exactly at leading order) and the
    interior rows' O((k h)^2).  A wrong sign of i k, or a missing factor, leaves
    an O(1/(k h)) boundary residual instead."""
    k = 20.0
    res = [_plane_wave_residual(n, k) for n in (200, 400, 800)]
    for n, (rb, ri) in zip((200, 400, 800), res):
        kh = k / n
        assert rb == pytest.approx(kh / 12, rel=0.1)
        assert ri < kh ** 2
    assert res[0][0] / res[1][0] == pytest.approx(2.0, rel=0.05)
    assert res[1][0] / res[2][0] == pytest.approx(2.0, rel=0.05)


def _mixed(ni=(14, 9), seed=3, c=None):
    g = I.Grid(2, ni, 0)
    if c is None:
        c = I.layered_grf(g, seed=seed, corr_cells=3.0)
    p = I.paper_params(g, c, ppw=10.0)
    P = oracle.Problem.from_grid(g, c, p, bc=I.MARMOUSI_BC)
    return g, c, p, P


def test_mixed_operator_eigenvalues_have_nonnegative_imaginary_parts():
    """Sec. 4: with a sound-hard top and absorbing sides and bottom, every
    eigenvalue of A has Im >= 0; the shift moves them up by omega^2 s / c^2."""
    g, c, p, P = _mixed()
    lam = np.linalg.eigvals(P.dense())
    assert lam.imag.min() >= -1e-9 * np.abs(lam).max()
    lam_s = np.linalg.eigvals(P.dense(shifted=True))
    assert lam_s.imag.min() >= p.omega ** 2 * p.shift / c.max() ** 2 * (1 - 1e-9)


def test_mixed_operator_is_complex_symmetric():
    """Ghost points only change diagonal entries, so A = A^T still holds."""
    _, _, _, P = _mixed(seed=5)
    A = P.dense()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()


def test_dirichlet_default_is_unchanged_by_explicit_faces():
    g = I.Grid(2, (10, 8), 3)
    c = I.layered_grf(g, seed=7, corr_cells=3.0)
    p = I.paper_params(g, c, ppw=10.0)
    P0 = oracle.Problem.from_grid(g, c, p)
    P1 = oracle.Problem.from_grid(g, c, p, bc=["dirichlet"] * 4)
    x = I.random_complex(g.n_total, 1)
    assert np.array_equal(P0.apply(x), P1.apply(x))


def test_fgmres_with_mixed_faces_reaches_the_direct_solution():
    g, c, p, P = _mixed(ni=(40, 12), seed=9)
    b = I.rhs_from_source(I.gaussian_source(g, center=(0.5, 2.5 / 40))).ravel()
    u, info = P.fgmres(b, rtol=1e-8, maxit=400)
    assert info["converged"] and info["true_relres"] <= 1e-8
    ref = np.linalg.solve(P.dense(), b)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-6
