"""Pins for the oracle's cell mass matrix (element-local L2 inner product of Sec. 5.1).

* exact integration: 1^T M x of an interpolated Q_k polynomial equals its
  exact integral over the box (the Gauss rule is exact to degree 2k+1);
* M_e is the exact Gram matrix of the basis: a (k+4)-point Gauss rule gives
  the same matrix;
* tensor-product structure and DoF layout: M_e = det J (M1 (x) M1 (x) M1) per
  component, with M1 built here from numpy's Legendre-Gauss rule and the
  Lagrange basis written out;
* symmetric positive definite, and the inverse undoes it.
"""
import numpy as np
import pytest

from oracle import mass
from oracle.mesh import BoxMesh
from oracle.sipg import SIPG


@pytest.mark.parametrize("k", [1, 2, 4])
def test_integral_of_interpolated_polynomial(k):
    mesh = BoxMesh(3, 2, 2, extent=(1.5, 1.0, 0.5))
    S = SIPG(mesh, k, 1)
    a, b, c = k, min(1, k), k  # x^a y^b z^c is in Q_k
    p = S.interpolate(lambda x: x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c)
    exact = 1.5 ** (a + 1) / (a + 1) * 1.0 ** (b + 1) / (b + 1) * 0.5 ** (c + 1) / (c + 1)
    assert abs(np.sum(mass.apply_mass(S, p)) - exact) <= 1e-14 * abs(exact) * 10


@pytest.mark.parametrize("k,ncomp", [(2, 3), (3, 1)])
def test_gram_matrix_exact(k, ncomp):
    mesh = BoxMesh(2, 1, 1, extent=(0.7, 0.3, 0.4))
    lo = mass.mass_block(SIPG(mesh, k, ncomp))
    hi = mass.mass_block(SIPG(mesh, k, ncomp, n_quad=k + 4))
    assert np.abs(lo - hi).max() <= 1e-14 * np.abs(hi).max()


def _lagrange(nodes, x):
    v = np.ones((len(x), len(nodes)))
    for j, xj in enumerate(nodes):
        for m, xm in enumerate(nodes):
            if m != j:
                v[:, j] *= (x - xm) / (xj - xm)
    return v


@pytest.mark.parametrize("k", [2, 3])
def test_tensor_product_structure(k):
    h = np.array([0.5, 0.25, 0.2])
    mesh = BoxMesh(2, 4, 5)
    S = SIPG(mesh, k, 3)
    t, w = np.polynomial.legendre.leggauss(2 * k + 4)
    t, w = 0.5 * (t + 1.0), 0.5 * w
    phi = _lagrange(S.nodes, t)
    M1 = np.einsum('q,qi,qj->ij', w, phi, phi)
    block = np.prod(h) * np.kron(np.kron(M1, M1), M1)   # index iz*n^2 + iy*n + ix
    M = mass.mass_block(S)
    n3 = (k + 1) ** 3
    for c in range(3):
        assert np.abs(M[c * n3:(c + 1) * n3, c * n3:(c + 1) * n3] - block).max() <= 1e-15 * 50
    assert np.abs(M[:n3, n3:]).max() == 0.0


def test_spd_and_inverse():
    mesh = BoxMesh(2, 2, 1)
    S = SIPG(mesh, 3, 3)
    M = mass.mass_block(S)
    assert np.abs(M - M.T).max() <= 1e-16
    assert np.linalg.eigvalsh(M).min() > 0
    x = np.random.default_rng(0).standard_normal(S.n_dofs)
    y = mass.apply_inverse_mass(S, mass.apply_mass(S, x, 2.5), 2.5)
    assert np.abs(y - x).max() <= 1e-12
