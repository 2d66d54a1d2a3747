"""Pins for the oracle's Helmholtz operator (Eq. helmholtz, Eq. pml-1d-s, Sec. 3.4 shift).

Each check compares against something other than the oracle's own formula:
a textbook closed form, the continuous PDE, a structural invariant, or a
property the paper states."""
import math

import numpy as np
import pytest

import oracle


def _sine_mode(shape_xyz, modes):
    u = np.ones(1)
    for n, a in zip(shape_xyz, modes):   # x first; numpy order needs reversing
        u = np.multiply.outer(np.sin(math.pi * a * (np.arange(n) + 1) / (n + 1)), u)
    return u.ravel()  # outer-product order gives [z][y][x] flattening (x fastest)


@pytest.mark.parametrize("dim,ni,modes", [(2, (9, 7), (1, 1)), (2, (9, 7), (4, 6)),
                                          (3, (5, 6, 4), (2, 1, 3))])
@pytest.mark.parametrize("shifted", [False, True])
def test_sine_modes_are_eigenvectors_without_pml(dim, ni, modes, shifted):
    """Dirichlet 3-point Laplacian: sin(pi a (j+1)/(n+1)) has eigenvalue
    -(4/h^2) sin^2(pi a / (2(n+1))) per axis (textbook closed form)."""
    omega, s = 3.7, 0.21
    c = np.ones(int(np.prod(ni)))
    P = oracle.Problem(dim, ni, 0, c, omega, s, 0.01)
    h = 1.0 / max(ni)
    u = _sine_mode(ni, modes)
    lam = omega ** 2 * (1 + 1j * s * shifted)
    for n, a in zip(ni, modes):
        lam -= 4.0 / h ** 2 * math.sin(math.pi * a / (2 * (n + 1))) ** 2
    Au = P.apply(u, shifted=shifted)
    assert np.allclose(Au, lam * u, rtol=0, atol=1e-10 * abs(lam))


def _cont_pml_1d(x, ux, uxx, L, delta, omega, C):
    """Continuous (1/s) d/dx ((1/s) du/dx) = u''/s^2 - s' u'/s^3 with the
    stretch of Eq. pml-1d-s."""
    alpha = C / (delta * omega)
    d = np.where(x < 0, -x, np.where(x > L, x - L, 0.0))
    dd = np.where(x < 0, -1.0, np.where(x > L, 1.0, 0.0))
    s = 1 + 1j * alpha * (d / delta) ** 2
    sp = 2j * alpha * d * dd / delta ** 2
    return uxx / s ** 2 - sp * ux / s ** 3


def _manufactured_error(N, omega=9.0, C=20.0):
    h = 1.0 / N
    p = N // 4
    delta = p * h
    n = N + 2 * p
    x = (np.arange(n) - p + 0.5) * h
    lo, hi = -delta - h / 2, 1 + delta + h / 2          # where the zero ghosts sit
    kx, ky = math.pi / (hi - lo), 2 * math.pi / (hi - lo)
    X, Xx, Xxx = np.sin(kx * (x - lo)), kx * np.cos(kx * (x - lo)), -kx ** 2 * np.sin(kx * (x - lo))
    Y, Yy, Yyy = np.sin(ky * (x - lo)), ky * np.cos(ky * (x - lo)), -ky ** 2 * np.sin(ky * (x - lo))
    c = 1.0 + 0.3 * np.outer(np.cos(3 * x), np.sin(2 * x))        # [y][x]
    P = oracle.Problem(2, (N, N), p, c, omega, 0.0, 1.0, C)
    U = np.outer(Y, X)
    AU = P.apply(U.ravel()).reshape(n, n)
    exact = (np.outer(Y, _cont_pml_1d(x, Xx, Xxx, 1.0, delta, omega, C))
             + np.outer(_cont_pml_1d(x, Yy, Yyy, 1.0, delta, omega, C), X)
             + omega ** 2 / c ** 2 * U)
    e = np.abs(AU - exact)
    return e.max(), np.sqrt(np.mean(e ** 2))


def test_pml_operator_converges_to_continuous_pml_operator():
    """Manufactured solution through the PML: the discrete operator converges at
    second order to the continuous stretched operator of Eq. pml-1d-s."""
    e64 = _manufactured_error(64)
    e128 = _manufactured_error(128)
    assert e64[0] / e128[0] > 3.5
    assert e64[1] / e128[1] > 3.5
    assert e128[1] < 0.05


@pytest.mark.parametrize("dim,ni,npml", [(2, (6, 8), 3), (3, (3, 4, 3), 2)])
def test_stretch_weighted_operator_is_complex_symmetric(dim, ni, npml):
    """prod_d s_d(x_p) * (A)_{pq} is complex symmetric: the flux form puts the
    same half-node factor on (p, p+e_d) and (p+e_d, p)."""
    rng = np.random.default_rng(3)
    n = tuple(m + 2 * npml for m in ni)
    c = 1.0 + 0.5 * rng.random(int(np.prod(n)))
    P = oracle.Problem(dim, ni, npml, c, 7.0, 0.1, 0.01)
    A = P.dense(shifted=True)
    h = 1.0 / max(ni)
    delta = npml * h
    alpha = 20.0 / (delta * 7.0)
    w = np.ones(1, dtype=complex)
    for d in range(dim):
        x = (np.arange(n[d]) - npml + 0.5) * h
        dist = np.maximum(0, np.maximum(-x, x - ni[d] * h))
        w = np.multiply.outer(1 + 1j * alpha * (dist / delta) ** 2, w)
    S = w.ravel()[:, None] * A
    assert np.allclose(S, S.T, rtol=1e-12, atol=1e-12 * np.abs(S).max())
    # and A itself is not symmetric when a PML is present
    assert not np.allclose(A, A.T, rtol=1e-6, atol=1e-6 * np.abs(A).max())


def test_pml_eigenvalues_in_upper_half_plane_and_shift_moves_them_up():
    """Sec. 3.3: with the PML all eigenvalues have Im >= 0; the complex shift of
    Sec. 3.4 adds i omega^2 s / c^2 and enlarges the gap to the real axis."""
    ni, npml = (14, 14), 5
    c = np.ones((ni[1] + 2 * npml) * (ni[0] + 2 * npml))
    omega = 2 * math.pi * 1.0 / (10 / 14)         # ppw 10
    P0 = oracle.Problem(2, ni, npml, c, omega, 0.0, 1.0)
    Ps = oracle.Problem(2, ni, npml, c, omega, 0.2, 1.0)
    ev0 = np.linalg.eigvals(P0.dense())
    evs = np.linalg.eigvals(Ps.dense(shifted=True))
    scale = np.abs(ev0).max()
    assert ev0.imag.min() > -1e-10 * scale
    assert evs.imag.min() > ev0.imag.min() + 0.5 * 0.2 * omega ** 2 * 0.9


def test_no_pml_operator_is_real_symmetric_for_real_medium():
    rng = np.random.default_rng(5)
    c = 1 + rng.random(6 * 5)
    P = oracle.Problem(2, (6, 5), 0, c, 4.0, 0.0, 1.0)
    A = P.dense()
    assert np.allclose(A.imag, 0)
    assert np.allclose(A, A.T)
