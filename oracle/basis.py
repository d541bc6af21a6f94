"""Lagrange polynomials on a node set (oracle, test infrastructure).

The shape functions of Q_k (Sec. 5) are tensor products of 1D Lagrange
polynomials l_j through the k+1 Gauss-Lobatto nodes:
  l_j(x) = prod_{m != j} (x - xi_m) / (xi_j - xi_m).
Derivatives use the product rule written out term by term.
Pinned in tests by partition of unity, the Kronecker property and exact
differentiation of polynomials of degree <= k.
"""
import numpy as np


def lagrange_values(nodes, x):
    """L[p, j] = l_j(x_p)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def lagrange_derivatives(nodes, x):
    """D[p, j] = l_j'(x_p)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((len(x), n))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[m]))
            for l in range(n):
                if l != j and l != m:
                    term *= (x - nodes[l]) / (nodes[j] - nodes[l])
            D[:, j] += term
    return D


def tensor_basis(nodes, xi):
    """Values and reference gradients of the 3D tensor-product basis.

    xi: (P, 3) reference points in [0,1]^3. Node index i = (iz*n + iy)*n + ix.
    Returns phi (P, n^3) and dphi (P, n^3, 3) with dphi[..., l] = d/dxi_l.
    """
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    n = len(nodes)
    Lx, Ly, Lz = (lagrange_values(nodes, xi[:, d]) for d in range(3))
    Dx, Dy, Dz = (lagrange_derivatives(nodes, xi[:, d]) for d in range(3))
    P = xi.shape[0]
    phi = np.einsum('pz,py,px->pzyx', Lz, Ly, Lx).reshape(P, n ** 3)
    g0 = np.einsum('pz,py,px->pzyx', Lz, Ly, Dx).reshape(P, n ** 3)
    g1 = np.einsum('pz,py,px->pzyx', Lz, Dy, Lx).reshape(P, n ** 3)
    g2 = np.einsum('pz,py,px->pzyx', Dz, Ly, Lx).reshape(P, n ** 3)
    return phi, np.stack([g0, g1, g2], axis=-1)
