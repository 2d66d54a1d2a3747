"""Host-side Taylor plan of the exp / psi actions (no GPU needed): the chosen
sub-step count and degree satisfy the remainder bound, respect the norm limit
per sub-step and the degree multiple, are the cheapest such choice in the
searched range, and the resulting polynomial reproduces the exponential of a
scalar of the bounded modulus in the left half plane (where the spectrum of
i t A_s lies) to the requested tolerance."""
import cmath
import math

import numpy as np
import pytest

from paper_2506_03617_gb300 import native as N

CASES = [(336.0, 1e-6, 4.0, 6), (160.0, 1e-6, 4.0, 4), (496.0, 1e-12, 6.0, 1), (40.0, 1e-12, 6.0, 8),
         (3.0, 1e-6, 4.0, 1), (1200.0, 1e-6, 4.0, 6)]


@pytest.fixture(scope="module")
def lib():
    try:
        return N.load()
    except Exception as e:
        pytest.skip(f"library unavailable: {e}")


def _log_bound(nu, S, m):
    th = nu / S
    return math.log(S) + (m + 1) * math.log(th) - math.lgamma(m + 2.0) + th


@pytest.mark.parametrize("case", CASES)
def test_plan_meets_the_bound_and_is_cheapest(lib, case):
    nu, tol, theta, kmult = case
    S, m = N.taylor_plan(nu, tol, theta, kmult)
    smin = max(1, math.ceil(nu / theta))
    assert S >= smin and m % kmult == 0
    assert _log_bound(nu, S, m) <= math.log(tol) + 1e-12
    best = min(S2 * m2 for S2 in range(smin, 4 * smin + 9)
               for m2 in range(kmult, 401, kmult) if _log_bound(nu, S2, m2) <= math.log(tol))
    assert S * m == best


@pytest.mark.parametrize("case", CASES[:4])
def test_plan_reproduces_the_scalar_exponential(lib, case):
    """(T_m(z/S))^S with T_m the degree-m Taylor polynomial equals e^z to the
    tolerance for |z| = nu, Re z <= 0."""
    nu, tol, theta, kmult = case
    S, m = N.taylor_plan(nu, tol, theta, kmult)
    for ang in np.linspace(math.pi / 2, 3 * math.pi / 2, 9):
        z = nu * cmath.exp(1j * ang)
        w = z / S
        t, term = 1.0 + 0j, 1.0 + 0j
        for k in range(1, m + 1):
            term *= w / k
            t += term
        approx = t ** S
        assert abs(approx - cmath.exp(z)) <= 10 * tol, (ang, abs(approx - cmath.exp(z)))


def test_invalid_arguments_are_rejected(lib):
    assert N.taylor_plan(-1.0, 1e-6, 4.0) is None
    assert N.taylor_plan(10.0, 0.0, 4.0) is None
    assert N.taylor_plan(10.0, 1e-6, 0.0) is None
    assert N.taylor_plan(10.0, 1e-6, 4.0, 0) is None
