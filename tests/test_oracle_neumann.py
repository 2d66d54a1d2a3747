"""Pin for the oracle's truncated Neumann preconditioner P_N (Sec. 3.2):
Thm. 3.1 -- P_N is a function of A, and -i t P_N A = I - exp(i (N+1) t A), so
its eigenvalues are 1 - exp(i (N+1) t lambda_k) and lie in the disk of radius
exp(-(N+1) t lambda*) around 1."""
import numpy as np

import oracle
from paper_2506_03617_gb300 import inputs as I


def test_eigenvalues_of_PN_A_follow_theorem_3_1():
    g = I.Grid(2, (8, 8), 2)
    c = I.layered_grf(g, seed=71, corr_cells=2.0)
    p = I.paper_params(g, c, ppw=10.0)
    P = oracle.Problem(2, g.ni, g.npml, c, p.omega, 0.0, p.t / 4)  # unshifted: P_N built from A
    A = P.dense(shifted=False)
    n = g.n_total
    N = 3
    M = np.empty((n, n), complex)
    e = np.zeros(n, complex)
    for j in range(n):
        e[j] = 1
        M[:, j] = P.neumann(e, N, shifted=False)
        e[j] = 0
    t = p.t / 4
    PNA = -1j * t * M @ A
    lam = np.linalg.eigvals(A)
    mu = np.linalg.eigvals(PNA)
    pred = 1 - np.exp(1j * (N + 1) * t * lam)
    # same multiset: every predicted eigenvalue has a computed one next to it and back
    d1 = np.abs(pred[:, None] - mu[None, :]).min(axis=1)
    d2 = np.abs(mu[:, None] - pred[None, :]).min(axis=1)
    assert d1.max() < 1e-8 and d2.max() < 1e-8
    lam_star = lam.imag.min()
    assert np.abs(mu - 1).max() <= np.exp(-(N + 1) * t * lam_star) + 1e-9
    # and the identity itself
    assert np.allclose(PNA, np.eye(n) - __import__("scipy.linalg").linalg.expm(1j * (N + 1) * t * A),
                       atol=1e-9)
