"""The quadrature tables the library derives on the host (its own Gauss-Newton
solution of the triangle rules' moment equations and its Golub-Welsch
Gauss-Legendre), pinned on the CPU by closed forms: exact monomial moments
over the reference triangle up to each rule's degree (int xi^i eta^j =
i! j! / (i + j + 2)!), positive weights and points inside, the triangle's
symmetry; Gauss-Legendre exact for x^k up to k = 2n - 1, symmetric about
1/2, and equal to NumPy's Gauss-Legendre."""

from math import factorial

import numpy as np
import pytest

from paper_2604_21181_gb300 import api


def _moment(i, j):
    return factorial(i) * factorial(j) / factorial(i + j + 2)


@pytest.mark.parametrize("q,deg", [(6, 4), (12, 6)])
def test_triangle_rules_are_exact_to_their_degree(q, deg):
    xi, eta, w = api.quadrature_rule(api.RULE_TRIANGLE, q)
    assert np.all(w > 0)
    assert np.all(xi > 0) and np.all(eta > 0) and np.all(xi + eta < 1)
    for i in range(deg + 1):
        for j in range(deg + 1 - i):
            assert abs(np.sum(w * xi ** i * eta ** j) - _moment(i, j)) <= 1e-15, (i, j)
    # not exact one degree higher (the rule is the one of the stated degree)
    err = max(abs(np.sum(w * xi ** i * eta ** (deg + 1 - i)) - _moment(i, deg + 1 - i))
              for i in range(deg + 2))
    assert err > 1e-8
    # invariant under the permutations of the barycentric coordinates
    bary = np.stack([1 - xi - eta, xi, eta], axis=1)
    key = {tuple(np.round(np.append(b, wt), 12)) for b, wt in zip(bary, w)}
    for perm in ([1, 2, 0], [2, 0, 1], [1, 0, 2]):
        assert {tuple(np.round(np.append(b[perm], wt), 12)) for b, wt in zip(bary, w)} == key


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16, 33, 64, 100, 512])
def test_gauss_legendre_on_the_unit_interval(n):
    x, _, w = api.quadrature_rule(api.RULE_GAUSS_LEGENDRE, n)
    assert np.all(np.diff(x) > 0) and x[0] > 0 and x[-1] < 1
    assert np.all(w > 0)
    # weights from squared eigenvector components: rounding-level absolute
    # error (about 1e-15 at n = 512), not relative, in the small tail weights
    assert np.allclose(x + x[::-1], 1.0, atol=2e-15, rtol=0)
    assert np.allclose(w, w[::-1], atol=2e-15, rtol=0)
    for k in range(min(2 * n - 1, 60) + 1):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) <= 2e-15 * max(1, n / 8), k
    if n <= 100:
        t, v = np.polynomial.legendre.leggauss(n)
        assert np.allclose(x, 0.5 * (t + 1), atol=1e-15, rtol=0)
        assert np.allclose(w, 0.5 * v, atol=2e-16 * n, rtol=1e-13)


def test_invalid_rule_requests():
    lib = api.load_library()
    a = np.zeros(16)
    p = a.ctypes.data_as(api.C.POINTER(api.C.c_double))
    assert lib.mueller_quadrature_rule(api.RULE_TRIANGLE, 7, p, p, p) == 1
    assert lib.mueller_quadrature_rule(api.RULE_TRIANGLE, 6, p, None, p) == 1
    assert lib.mueller_quadrature_rule(api.RULE_GAUSS_LEGENDRE, 0, p, None, p) == 1
    assert lib.mueller_quadrature_rule(api.RULE_GAUSS_LEGENDRE, 513, p, None, p) == 1
    assert lib.mueller_quadrature_rule(5, 6, p, p, p) == 1
    assert lib.mueller_quadrature_rule(api.RULE_GAUSS_LEGENDRE, 4, None, None, p) == 1


@pytest.mark.parametrize("q,deg", [(6, 4), (12, 6)])
def test_library_and_oracle_rules_agree(q, deg):
    """The library and the oracle each solve the triangle rule's moment
    equations on their own.  Both solutions are exact to the rule's degree,
    and they agree to 1e-13 in the points and 1e-12 in the weights.  The
    12-point solutions differ by about 5e-14 and 4e-13 there, because the
    degree-6 equations are ill-conditioned in the last digits; that is far
    inside the 1e-11 of the operator parity."""
    oracle = pytest.importorskip("oracle")
    xi, eta, w = api.quadrature_rule(api.RULE_TRIANGLE, q)
    xo, eo, wo = oracle.tri_rule(q)
    assert np.abs(xi - xo).max() <= 1e-13 and np.abs(eta - eo).max() <= 1e-13
    assert np.abs(w - wo).max() <= 1e-12 * w.max()
    for i in range(deg + 1):
        for j in range(deg + 1 - i):
            assert abs(np.sum(wo * xo ** i * eo ** j) - _moment(i, j)) <= 1e-15, (i, j)
