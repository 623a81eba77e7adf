"""Pins of the oracle's Jacobi polynomials and quadrature rules against
closed forms, textbook tables and an independent library (scipy)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.special as sp

from oracle import jacobi as J
from oracle import quadrature as Qd
from oracle.operators import reference

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n,a,b", [(0, 0, 0), (1, 1, 1), (3, 0, 0), (5, 1, 1), (4, 3, 1), (6, 5, 1), (7, 2, 0)])
def test_jacobi_matches_scipy(n, a, b):
    z = np.linspace(-1, 1, 17)
    np.testing.assert_allclose(J.jacobi(n, a, b, z), sp.eval_jacobi(n, a, b, z), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("n,a", [(3, 0), (4, 1), (6, 3), (5, 7)])
def test_jacobi_endpoint(n, a):
    # P_n^{(a,b)}(1) = binom(n + a, n)
    assert J.jacobi(n, a, 1.0, 1.0) == pytest.approx(math.comb(n + a, n), rel=1e-14)


@pytest.mark.parametrize("n,a,b", [(3, 1, 1), (6, 1, 1), (5, 2, 1), (8, 1, 1), (9, 2, 1)])
def test_jacobi_zeros_match_scipy(n, a, b):
    x_ref, _ = sp.roots_jacobi(n, a, b)
    np.testing.assert_allclose(Qd.jacobi_zeros(n, a, b), np.sort(x_ref), atol=1e-13)


def _parse(expr):
    return float(eval(expr, {"sqrt": math.sqrt}))


def test_gll_textbook_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "gll_lobatto_closed_forms.txt")) if l.strip() and l[0] != "#"]
    for Q in (3, 4, 5):
        x, w = Qd.gll(Q)
        ref = sorted([(_parse(r[1]), _parse(r[2])) for r in rows if int(r[0]) == Q])
        np.testing.assert_allclose(x, [t[0] for t in ref], atol=1e-14)
        np.testing.assert_allclose(w, [t[1] for t in ref], atol=1e-14)


def _exact_moment(k, alpha):
    """int_{-1}^{1} x^k (1 - x)^alpha dx, exact rational (x = 2t - 1, Beta integrals)."""
    tot = Fraction(0)
    for j in range(k + 1):
        beta = Fraction(math.factorial(j) * math.factorial(alpha), math.factorial(j + alpha + 1))
        tot += math.comb(k, j) * Fraction(2) ** j * Fraction(-1) ** (k - j) * beta
    return float(tot * Fraction(2) ** (alpha + 1))


@pytest.mark.parametrize("Q", [3, 4, 6, 8, 10, 12])
def test_gll_degree_of_exactness(Q):
    x, w = Qd.gll(Q)
    for k in range(2 * Q - 2):
        assert np.dot(w, x ** k) == pytest.approx(_exact_moment(k, 0), abs=1e-13)
    # and no more: x^(2Q-2) is not integrated exactly by a Lobatto rule
    assert abs(np.dot(w, x ** (2 * Q - 2)) - _exact_moment(2 * Q - 2, 0)) > 1e-10


@pytest.mark.parametrize("Q,alpha", [(3, 1), (4, 1), (6, 2), (8, 1), (10, 2), (12, 2)])
def test_grj_degree_of_exactness(Q, alpha):
    x, w = Qd.grj(Q, alpha)
    assert x[0] == -1.0 and x.max() < 1.0
    for k in range(2 * Q - 1):
        assert np.dot(w, x ** k) == pytest.approx(_exact_moment(k, alpha), abs=1e-12)
    assert abs(np.dot(w, x ** (2 * Q - 1)) - _exact_moment(2 * Q - 1, alpha)) > 1e-10


def _fact(n):
    return math.factorial(n)


def _ref_integral(shape, a, b, c):
    """Exact int over the reference element of xi1^a xi2^b xi3^c (t = (1+xi)/2)."""
    tot = Fraction(0)
    for i in range(a + 1):
        for j in range(b + 1):
            for k in range(c + 1):
                coef = (math.comb(a, i) * math.comb(b, j) * math.comb(c, k) * Fraction(2) ** (i + j + k)
                        * Fraction(-1) ** (a - i + b - j + c - k))
                if shape == 0:
                    m = Fraction(1, (i + 1) * (j + 1) * (k + 1))
                elif shape == 1:     # t1 + t3 <= 1, t2 in [0,1]
                    m = Fraction(_fact(i) * _fact(k), _fact(i + k + 2)) * Fraction(1, j + 1)
                elif shape == 2:     # t1, t2 <= 1 - t3
                    m = Fraction(_fact(k) * _fact(i + j + 2), _fact(i + j + k + 3) * (i + 1) * (j + 1))
                else:                # simplex (Dirichlet integral)
                    m = Fraction(_fact(i) * _fact(j) * _fact(k), _fact(i + j + k + 3))
                tot += coef * m
    return float(tot * 8)


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
@pytest.mark.parametrize("Q", [3, 5])
def test_3d_rules_integrate_polynomials(shape, Q):
    ref = reference(shape, 1, Q)
    xi, W = ref["xi"], ref["W"]
    deg = 2 * Q - 3
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                val = np.dot(W, xi[0] ** a * xi[1] ** b * xi[2] ** c)
                assert val == pytest.approx(_ref_integral(shape, a, b, c), abs=1e-12), (a, b, c)


@pytest.mark.parametrize("shape,vol", [(0, 8.0), (1, 4.0), (2, 8.0 / 3.0), (3, 4.0 / 3.0)])
def test_reference_volumes(shape, vol):
    for Q in (3, 6, 10):
        assert reference(shape, 1, Q)["W"].sum() == pytest.approx(vol, rel=1e-14)
