"""Pins for oracle/gll.py: closed forms, quadrature exactness, library roots."""
import os

import numpy as np
import pytest

from oracle.gll import (gll_nodes_weights, derivative_matrix, lagrange_basis,
                        lagrange_basis_derivative)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        n, i, t, w = line.split()
        ns = {"sqrt": np.sqrt}
        rows.setdefault(int(n), []).append((eval(t, ns), eval(w, ns)))
    return rows


def test_closed_forms():
    for n, vals in _golden().items():
        t, rho = gll_nodes_weights(n)
        np.testing.assert_allclose(t, [v[0] for v in vals], rtol=0, atol=1e-15)
        np.testing.assert_allclose(rho, [v[1] for v in vals], rtol=1e-14)


@pytest.mark.parametrize("n", range(1, 10))
def test_quadrature_exactness(n):
    t, rho = gll_nodes_weights(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(rho * t ** k) - exact) < 1e-13
    # GLL is not exact at degree 2n (this separates it from Gauss points)
    k = 2 * n
    assert abs(np.sum(rho * t ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("n", range(2, 10))
def test_nodes_are_roots_of_legendre_derivative(n):
    t, _ = gll_nodes_weights(n)
    roots = np.sort(np.polynomial.legendre.Legendre.basis(n).deriv().roots().real)
    np.testing.assert_allclose(t[1:-1], roots, atol=1e-13)


@pytest.mark.parametrize("n", range(1, 10))
def test_derivative_matrix(n):
    t, _ = gll_nodes_weights(n)
    D = derivative_matrix(n)
    # closed form == term-by-term derivative of the product-formula basis
    np.testing.assert_allclose(D, lagrange_basis_derivative(t, t), atol=1e-12 * n * n)
    # exact on polynomials of degree <= n
    for k in range(n + 1):
        d_exact = k * t ** (k - 1) if k > 0 else 0 * t
        np.testing.assert_allclose(D @ t ** k, d_exact, atol=1e-12 * n * n)
    np.testing.assert_allclose(D.sum(axis=1), 0, atol=1e-12 * n * n)
    # basis is cardinal on the nodes
    np.testing.assert_allclose(lagrange_basis(t, t), np.eye(n + 1), atol=1e-14)
