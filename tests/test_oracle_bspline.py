"""Pins of the oracle's temporal basis against the paper and exact arithmetic.

- Table 1 (Section 2.3) for w^{kappa,d} (golden fixture).
- B-spline values against the Cox-de Boor recursion in exact rational
  arithmetic (a different definition of the same spline than Eq. decompose).
- Partition of unity, support (Remark support), symmetry, the maximum of
  N^{0,2} (3/4) and the discrete moments of the cardinal B-spline.
- Derivative and integral against finite differences / quadrature.
"""

import os
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import coeffs as oc

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = {}
    for line in open(os.path.join(GOLD, "table1_w.txt")):
        if line.startswith("#") or not line.strip():
            continue
        d, vals = line.split(":")
        rows[int(d)] = [F(v) for v in vals.split()]
    return rows


def test_w_matches_table1():
    for d, vals in _table1().items():
        assert len(vals) == d + 2
        for k, v in enumerate(vals):
            assert oc.w(k, d) == pytest.approx(float(v), abs=1e-15)


def _cox_de_boor(d, t):
    """N^{0,d}(t) on knots 0..d+1 by the Cox-de Boor recursion, exact."""
    t = F(t)

    def N(i, e):
        if e == 0:
            return F(1) if i <= t < i + 1 else F(0)
        return ((t - i) * N(i, e - 1) + (i + e + 1 - t) * N(i + 1, e - 1)) / e

    return N(0, d)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_N_against_cox_de_boor(d):
    for t in [F(1, 7), F(1, 3), F(1, 2), F(2, 3), F(5, 4), F(3, 2), F(9, 5), F(21, 10), F(13, 5), F(31, 9)]:
        if t >= d + 1:
            continue
        assert oc.N(d, float(t)) == pytest.approx(float(_cox_de_boor(d, t)), abs=2e-16)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_partition_of_unity_support_symmetry(d):
    for x in np.linspace(0.0, 1.0, 13)[:-1]:
        s = sum(oc.N(d, x + j) for j in range(-1, d + 2))
        assert s == pytest.approx(1.0, abs=1e-15)
    assert oc.N(d, 0.0) == 0.0 and oc.N(d, -0.3) == 0.0
    assert oc.N(d, d + 1.0) == 0.0 and oc.N(d, d + 1.7) == 0.0
    for x in np.linspace(0.05, d + 0.95, 17):
        assert oc.N(d, x) == pytest.approx(oc.N(d, d + 1 - x), abs=1e-15)
        assert oc.N(d, x) > 0


def test_quadratic_bspline_maximum():
    xs = np.linspace(0, 3, 3001)
    assert max(oc.N(2, x) for x in xs) == pytest.approx(0.75, abs=1e-15)
    assert oc.N(2, 1.5) == pytest.approx(0.75, abs=1e-15)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_discrete_moments(d):
    # sum_j (x + j) N(x + j) = (d+1)/2 for d >= 1 and
    # sum_j (x + j)^2 N(x + j) = ((d+1)/2)^2 + (d+1)/12 for d >= 2
    m, v = (d + 1) / 2.0, (d + 1) / 12.0
    for x in (0.1, 0.37, 0.8):
        taus = [x + j for j in range(0, d + 1)]
        m1 = sum(t * oc.N(d, t) for t in taus)
        assert m1 == pytest.approx(m, abs=1e-14)
        if d >= 2:
            m2 = sum(t * t * oc.N(d, t) for t in taus)
            assert m2 == pytest.approx(m * m + v, abs=1e-14)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_derivative_and_integral(d):
    h = 1e-6
    for x in np.linspace(0.013, d + 0.987, 24):
        fd = (oc.N(d, x + h) - oc.N(d, x - h)) / (2 * h)
        assert oc.dN(d, x) == pytest.approx(fd, abs=1e-8)
        gd = (oc.G(d, x + h) - oc.G(d, x - h)) / (2 * h)
        assert gd == pytest.approx(oc.N(d, x), abs=1e-8)
        assert oc.G(d, x) + oc.Gc(d, x) == pytest.approx(1.0, abs=1e-15)
    assert oc.G(d, d + 1.0) == 1.0 and oc.G(d, 0.0) == 0.0
    # left limits of the derivative at knots (d = 1: the hat function)
    if d == 1:
        assert oc.dN(1, 1.0) == 1.0 and oc.dN(1, 2.0) == -1.0 and oc.dN(1, 0.0) == 0.0
