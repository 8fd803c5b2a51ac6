"""Pins of the oracle's GLL basis (Section 2) against closed forms and exactness."""
import json
import os

import numpy as np
import pytest

from oracle.gll import diff_matrix, gll_nodes, gll_weights, lagrange_eval

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.json")))


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_closed_forms(P):
    rule = GOLD["rules"][str(P)]
    np.testing.assert_allclose(gll_nodes(P), rule["nodes"], atol=1e-15)
    np.testing.assert_allclose(gll_weights(P), rule["weights"], rtol=1e-14)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 8, 16, 32])
def test_quadrature_exact_to_degree_2p_minus_1(P):
    x, w = gll_nodes(P), gll_weights(P)
    for k in range(2 * P):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13, (P, k)
    # not exact at degree 2P: the rule integrates L_P^2 to 2/P instead of 2/(2P+1)
    c = np.zeros(P + 1)
    c[P] = 1.0
    lp = np.polynomial.legendre.legval(x, c)
    assert abs(np.dot(w, lp ** 2) - 2.0 / P) < 1e-12
    assert abs(np.dot(w, lp ** 2) - 2.0 / (2 * P + 1)) > 0.1 / P


@pytest.mark.parametrize("P", [1, 2, 4, 8, 16, 32])
def test_nodes_symmetric_and_sorted(P):
    x = gll_nodes(P)
    assert np.all(np.diff(x) > 0)
    np.testing.assert_allclose(x, -x[::-1], atol=1e-15)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 8, 16])
def test_diff_matrix_exact_on_polynomials(P):
    x = gll_nodes(P)
    D = diff_matrix(x)
    rng = np.random.default_rng(P)
    c = rng.standard_normal(P + 1)
    p = np.polynomial.Polynomial(c)
    tol = 1e-13 * (P + 1) ** 2 * np.abs(c).sum()
    assert np.max(np.abs(D @ p(x) - p.deriv()(x))) < tol
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-12 * (P + 1) ** 2)


@pytest.mark.parametrize("Pc,Pf", [(1, 2), (2, 4), (4, 8), (8, 16), (16, 32)])
def test_lagrange_interpolation_exact(Pc, Pf):
    xc, xf = gll_nodes(Pc), gll_nodes(Pf)
    phi = lagrange_eval(xc, xf)
    np.testing.assert_allclose(lagrange_eval(xc, xc), np.eye(Pc + 1), atol=1e-13)
    rng = np.random.default_rng(Pf)
    p = np.polynomial.Polynomial(rng.standard_normal(Pc + 1))
    np.testing.assert_allclose(phi @ p(xc), p(xf), atol=1e-11)
    np.testing.assert_allclose(phi.sum(axis=1), 1.0, atol=1e-12)
