"""Pins of the oracle's quadrature rules and Sauter-Schwab maps (Sec. 4.2, 5.1).

Every rule is checked against what mathematics fixes: exactness on
monomials (triangle rules: a!b!/(a+b+2)!), agreement with NumPy's
Gauss-Legendre, and exact integration of polynomials over T x T by the
Sauter-Schwab point sets of all three classes (a wrong sub-region, Jacobian
or coordinate map fails one of these)."""

import math

import numpy as np
import pytest

import oracle


def simplex_moment(a, b):
    # int over {xi, eta >= 0, xi + eta <= 1} of xi^a eta^b
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


@pytest.mark.parametrize("q,deg", [(6, 4), (12, 6)])
def test_triangle_rule_exact_to_degree(q, deg):
    xi, eta, w = oracle.tri_rule(q)
    assert len(w) == q
    assert np.all(w > 0)
    assert np.all(xi >= 0) and np.all(eta >= 0) and np.all(xi + eta <= 1)
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            got = np.sum(w * xi ** a * eta ** b)
            assert abs(got - simplex_moment(a, b)) < 2e-15, (q, a, b)


@pytest.mark.parametrize("q,deg", [(6, 4), (12, 6)])
def test_triangle_rule_not_exact_beyond_degree(q, deg):
    # a rule of degree d fails on some monomial of degree d+1 (sanity: the
    # previous test is not vacuous)
    xi, eta, w = oracle.tri_rule(q)
    errs = [abs(np.sum(w * xi ** a * eta ** (deg + 1 - a)) - simplex_moment(a, deg + 1 - a))
            for a in range(deg + 2)]
    assert max(errs) > 1e-8


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 12, 20])
def test_gauss_legendre_matches_numpy(n):
    x, w = oracle.gauss_legendre01(n)
    t, v = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, 0.5 * (t + 1), atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * v, atol=1e-15)


def tri_ss_moment(a, b):
    # int over T^ = {0 <= v <= u <= 1} of u^a v^b
    return 1.0 / ((b + 1) * (a + b + 2))


@pytest.mark.parametrize("cls,nreg", [(3, 6), (2, 5), (1, 2)])
def test_sauter_schwab_points_cover_pair_domain(cls, nreg):
    ns = 6
    P = oracle.ss_points(cls, ns)
    assert P.shape == (nreg * ns ** 4, 5)
    xu, xv, yu, yv, w = P.T
    tol = 1e-15
    assert np.all((xv >= -tol) & (xv <= xu + tol) & (xu <= 1 + tol))
    assert np.all((yv >= -tol) & (yv <= yu + tol) & (yu <= 1 + tol))
    assert np.all(w > 0)
    # every class integrates any polynomial over T^ x T^ exactly
    rng = np.random.default_rng(7)
    for _ in range(25):
        a, b, c, d = rng.integers(0, 3, size=4)
        got = np.sum(w * xu ** a * xv ** b * yu ** c * yv ** d)
        ref = tri_ss_moment(a, b) * tri_ss_moment(c, d)
        assert abs(got - ref) < 1e-14, (cls, a, b, c, d, got, ref)
    # mixed terms couple x and y: (u_x - u_y)^2 (v_x - v_y)^2
    got = np.sum(w * (xu - yu) ** 2 * (xv - yv) ** 2)
    ref = 0.0
    for i in range(3):
        for j in range(3):
            ci = math.comb(2, i) * (-1) ** (2 - i)
            cj = math.comb(2, j) * (-1) ** (2 - j)
            ref += ci * cj * tri_ss_moment(i, j) * tri_ss_moment(2 - i, 2 - j)
    assert abs(got - ref) < 1e-14


def test_sauter_schwab_singular_point_is_where_expected():
    # coincident: x == y on the diagonal xi-measure zero; edge: shared points
    # have v = 0 in both; vertex: (0,0).  The Jacobian weights vanish there.
    for cls in (1, 2, 3):
        P = oracle.ss_points(cls, 4)
        d = np.hypot(P[:, 0] - P[:, 2], P[:, 1] - P[:, 3])
        assert d.min() > 0.0  # Gauss points never hit the singular set
