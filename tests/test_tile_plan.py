"""Host-side tile planner of the persistent exp kernel (no GPU needed): every
plan covers the grid, fits the co-resident CTAs and the per-CTA region, keeps
all tiles but the last of each axis at least K cells wide (so a tile's K-cell
ring lies inside its eight neighbours, the only tiles a pass waits for), and
has the smallest region per CTA among all such splits (brute force)."""
import itertools

import pytest

from paper_2506_03617_gb300 import native as N

CASES = [(52, 48, 152, 4, 88, 104), (11, 48, 152, 4, 88, 104), (1088, 1088, 152, 4, 88, 104),
         (302, 169, 152, 2, 124, 68), (84, 84, 152, 2, 124, 68), (3, 3, 152, 4, 88, 104),
         (4000, 7, 152, 4, 88, 104), (500, 500, 40, 4, 88, 104), (1, 1, 1, 2, 8, 8)]


@pytest.fixture(scope="module")
def lib():
    try:
        return N.load()
    except Exception as e:  # the library is built by build(); nvcc may be absent
        pytest.skip(f"library unavailable: {e}")


def _ceil(a, b):
    return -(-a // b)


def _admissible(n0, n1, slots, k, txmax, tymax, a, b):
    ntx, nty = _ceil(n0, a), _ceil(n1, b)
    return (a <= txmax and b <= tymax and ntx * nty <= min(slots, 4096)
            and (a >= k or ntx == 1) and (b >= k or nty == 1))


@pytest.mark.parametrize("case", CASES)
def test_plan_is_valid_and_minimal(lib, case):
    n0, n1, slots, k, txmax, tymax = case
    plan = N.persist_tile_plan(*case)
    assert plan is not None
    a, b, ntx, nty = plan
    assert ntx == _ceil(n0, a) and nty == _ceil(n1, b)
    assert (ntx - 1) * a < n0 <= ntx * a and (nty - 1) * b < n1 <= nty * b
    assert _admissible(n0, n1, slots, k, txmax, tymax, a, b)
    best = min((a2 + 2 * k) * (b2 + 2 * k)
               for a2, b2 in itertools.product(range(1, min(n0, txmax) + 1), range(1, min(n1, tymax) + 1))
               if _admissible(n0, n1, slots, k, txmax, tymax, a2, b2))
    assert (a + 2 * k) * (b + 2 * k) == best


def test_plan_refuses_grids_that_do_not_fit(lib):
    assert N.persist_tile_plan(1088, 1088, 10, 4, 88, 104) is None      # needs 13 x 11 tiles
    assert N.persist_tile_plan(0, 10, 152, 4, 88, 104) is None
    assert N.persist_tile_plan(10, 10, 152, 0, 88, 104) is None
