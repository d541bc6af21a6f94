"""Element mass matrices and their inverses (oracle, test infrastructure).

The element-local L2 inner product (v, u)_{Omega_e} appears in every step of
the splitting scheme of Sec. 5.1: it is the left-hand side of the convective
step, Eq. (convective_step_weak), of the velocity projection step,
Eq. (projection_step_weak), and the gamma_0/dt term of the viscous step,
Eq. (viscous_step_weak). With a discontinuous space it couples only the
coefficients of one cell, so "a simple mass matrix solve" (Sec. 3.2, below
Eq. convective_step) is a solve with one small block per cell.

The oracle builds each block literally as
    M_e[a, b] = sum_q w_q det J  phi_a(xi_q) . phi_b(xi_q)
with the cell's k+1 point Gauss rule and the vector basis phi_a = phi_i e_c,
then multiplies (or solves with numpy's dense solver) cell by cell. On the
affine box map all cells share one block up to nothing (equal cells), but the
oracle does not use that.

Pins (tests/test_oracle_mass.py): 1^T M x equals the exact integral of the
interpolated polynomial (degree <= k, Gauss is exact to 2k+1); the block of
constants sums to the cell volume; M is symmetric positive definite; M^-1 M x
= x; the tensor-product structure M_e = det J (M1 (x) M1 (x) M1) per component
against a 1D matrix computed by brute-force quadrature with more points.
"""
import numpy as np


def mass_block(sipg, e=0):
    """M_e of operator ``sipg`` (an affine SIPG or a trilinear MappedSIPG space; its
    ncomp picks vector or scalar). On trilinear cells the weights are w_q det J(xi_q)."""
    if hasattr(sipg, 'cell_geometry'):
        W = sipg.cell_geometry(e)[2]
    else:
        W = sipg.cell_w * sipg.mesh.volume()
    phi = sipg.cell_phi
    if sipg.ncomp == 1:
        return np.einsum('q,qa,qb->ab', W, phi, phi)
    V, _ = sipg._vector_basis(phi, np.zeros(phi.shape + (3,)))
    return np.einsum('q,qak,qbk->ab', W, V, V)


def apply_mass(sipg, x, coeff=1.0):
    """y = coeff M x, cell by cell."""
    m = sipg.n_dofs_cell
    X = np.asarray(x, dtype=np.float64).reshape(sipg.mesh.n_cells, m)
    Y = np.empty_like(X)
    for e in range(sipg.mesh.n_cells):
        Y[e] = coeff * (mass_block(sipg, e) @ X[e])
    return Y.reshape(-1)


def apply_inverse_mass(sipg, x, coeff=1.0):
    """y = (coeff M)^-1 x, one dense solve per cell."""
    m = sipg.n_dofs_cell
    X = np.asarray(x, dtype=np.float64).reshape(sipg.mesh.n_cells, m)
    Y = np.empty_like(X)
    for e in range(sipg.mesh.n_cells):
        Y[e] = np.linalg.solve(coeff * mass_block(sipg, e), X[e])
    return Y.reshape(-1)
