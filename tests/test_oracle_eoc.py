"""Pin of the oracle's discretisation against the paper's EOC table.

Section 3.4 (Table gridrefinementerr) runs the scheme with G = 1, no rescaling
and the exact solution u = (|x|^2 - 1)/6 + t as Dirichlet data.  That exercises
the reduced diamond-cell gradient, A_eps on faces, Abar per voxel, the
semi-implicit system (Eq. new), the SOR solve and the ghost-cell boundary
handling at once: a dropped tangential term, a wrong Abar average or a wrong
power of h changes the order of convergence.

Reading: the table labels its runs "eps = h^2"; its orders are reproduced
when h^2 is the quantity added under the square root, i.e. eps = h in the
notation of Eq. 3rd.  With that reading the EOC column is matched to within
0.05, and no other multiple of h does that (0.5 h, 2 h, 3 h and 6 h give
orders 2.26/2.13, 1.39/1.61, 1.09/1.34, 0.70/0.80).  The absolute errors
come out a near-constant factor of 2.41-2.48 below the printed ones (same
shape).  Neither the final-time L2 norm nor the root of the summed per-step
norms reproduces the printed values, and rescaling u by the 1/6 of the exact
solution is equivalent to eps/6, which breaks the orders; so absolute values
are pinned only up to that constant.
"""
import math
import os

import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eoc_table.txt")


def _table():
    rows = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            n, h, steps, err, eoc = line.split()
            rows[int(n)] = (float(h), int(steps), float(err), None if eoc == "-" else float(eoc))
    return rows


def _run(n):
    table = _table()
    h, steps, _, _ = table[n]
    assert abs(h - 2.5 / n) < 1e-15
    # eps = h: h^2 is what is added under the square root
    err, info = O.eoc(n, steps, T=0.0625, L=1.25, eps_factor=1.0 / h, omega=1.5, tol=1e-12)
    assert info["status"] == O.OR_OK
    return err


@pytest.fixture(scope="module")
def errs():
    return {n: _run(n) for n in (10, 20, 40)}


def test_eoc_orders_match_table(errs):
    table = _table()
    for coarse, fine in ((10, 20), (20, 40)):
        eoc = math.log2(errs[coarse] / errs[fine])
        assert abs(eoc - table[fine][3]) < 0.05, (coarse, fine, eoc, table[fine][3])


def test_eoc_absolute_errors_same_shape(errs):
    table = _table()
    ratios = [table[n][2] / errs[n] for n in (10, 20, 40)]
    # a constant normalisation factor, not a different error curve
    assert all(2.2 < r < 2.7 for r in ratios), ratios
    assert max(ratios) / min(ratios) < 1.05, ratios


def test_eoc_literal_eps_is_not_second_order():
    """The literal eps = h^2 reading gives a very different curve (guards the
    reading above against silent drift)."""
    e10, _ = O.eoc(10, 1, eps_factor=1.0)
    e20, _ = O.eoc(20, 4, eps_factor=1.0)
    assert math.log2(e10 / e20) > 3.0
