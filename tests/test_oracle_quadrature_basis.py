"""Pins for the oracle's quadrature rules and Lagrange basis (no GPU)."""
import numpy as np
import pytest

from oracle import basis, quadrature


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = quadrature.gauss_legendre(n)
    for p in range(2 * n):
        assert abs(np.sum(w * x ** p) - 1.0 / (p + 1)) < 1e-15
    # and not exact one degree higher (the rule is the n-point one)
    p = 2 * n
    assert abs(np.sum(w * x ** p) - 1.0 / (p + 1)) > 1e-12


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7])
def test_gauss_lobatto_exact_to_degree_2n_minus_3(n):
    x, w = quadrature.gauss_lobatto(n)
    assert x[0] == 0.0 and x[-1] == 1.0
    for p in range(2 * n - 2):
        assert abs(np.sum(w * x ** p) - 1.0 / (p + 1)) < 1e-15


def test_closed_form_nodes():
    x, w = quadrature.gauss_legendre(2)
    assert np.allclose(x, [0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)], atol=1e-16)
    assert np.allclose(w, [0.5, 0.5], atol=1e-16)
    x, w = quadrature.gauss_legendre(3)
    assert np.allclose(x, [0.5 - 0.5 * np.sqrt(0.6), 0.5, 0.5 + 0.5 * np.sqrt(0.6)], atol=1e-16)
    assert np.allclose(w, [5 / 18, 8 / 18, 5 / 18], atol=1e-16)
    x, w = quadrature.gauss_lobatto(3)
    assert np.allclose(x, [0, 0.5, 1], atol=1e-16) and np.allclose(w, [1 / 6, 4 / 6, 1 / 6], atol=1e-16)
    x, w = quadrature.gauss_lobatto(4)
    r = 0.5 / np.sqrt(5)
    assert np.allclose(x, [0, 0.5 - r, 0.5 + r, 1], atol=1e-16)
    assert np.allclose(w, [1 / 12, 5 / 12, 5 / 12, 1 / 12], atol=1e-16)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_lagrange_identities(k):
    nodes, _ = quadrature.gauss_lobatto(k + 1)
    L = basis.lagrange_values(nodes, nodes)
    assert np.allclose(L, np.eye(k + 1), atol=1e-14)
    xs = np.linspace(-0.2, 1.3, 17)
    assert np.allclose(basis.lagrange_values(nodes, xs).sum(axis=1), 1.0, atol=1e-12)
    assert np.allclose(basis.lagrange_derivatives(nodes, xs).sum(axis=1), 0.0, atol=1e-11)
    # exact derivative of every monomial of degree <= k
    for p in range(k + 1):
        d = basis.lagrange_derivatives(nodes, xs) @ nodes ** p
        exact = p * xs ** (p - 1) if p > 0 else 0 * xs
        assert np.allclose(d, exact, atol=1e-11)


def test_tensor_basis_gradient_by_finite_differences():
    nodes, _ = quadrature.gauss_lobatto(4)
    pt = np.array([[0.31, 0.62, 0.17]])
    phi, dphi = basis.tensor_basis(nodes, pt)
    h = 1e-6
    for l in range(3):
        e = np.zeros(3)
        e[l] = h
        fd = (basis.tensor_basis(nodes, pt + e)[0] - basis.tensor_basis(nodes, pt - e)[0]) / (2 * h)
        assert np.allclose(dphi[0, :, l], fd[0], atol=1e-8)
