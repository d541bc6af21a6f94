"""Continuous ("cph") multigrid levels below the DG level (oracle, test infrastructure).

Sec. 5.4: the hp-multigrid preconditioner first converts from the discontinuous
to a continuous polynomial space of the same degree, then lowers the degree,
then coarsens the mesh ("cph-multigrid", Fehn et al. 2020). On the box with
structured cells and Gauss-Lobatto nodes, the continuous space Q_k with C^0
continuity has one value per node of the global (nx k + 1) x (ny k + 1) x
(nz k + 1) grid and component; continuous functions enter the DG space through
the injection P (each cell copies the global values at its nodes).

* continuous level operator: the Galerkin product P^T A_DG P of the DG operator
  of the same mesh and degree (for continuous functions the interior-face
  terms of the SIPG form vanish, so this is the continuous-space form);
* DG -> continuous transfer: prolongation P, restriction P^T;
* continuous -> continuous transfers (degree or mesh): prolongation
  R_f Pdg P_c, where Pdg is the DG embedding of oracle.multigrid and R_f takes
  each fine global node's value from the lowest-index cell that holds it (all
  copies agree for the continuous fields it is applied to); restriction is its
  transpose.
Global numbering: component-major, node (gx, gy, gz) at (gz Gy + gy) Gx + gx.

Pins (tests/test_oracle_cph.py): P reproduces continuous polynomials exactly;
R P = I; the composed prolongation reproduces a continuous coarse polynomial
on the fine continuous level exactly (degree and mesh steps); the continuous
Galerkin operators are symmetric, definite with Dirichlet walls, and keep the
constants / rigid-body modes in their kernel with all-Neumann walls; the
continuous DoF count in closed form.
"""
import numpy as np
import scipy.sparse as sp

from . import multigrid as omg


def grid_dims(mesh, k):
    nx, ny, nz = mesh.n_cells_dir
    return nx * k + 1, ny * k + 1, nz * k + 1


def n_cg(mesh, k, ncomp):
    Gx, Gy, Gz = grid_dims(mesh, k)
    return ncomp * Gx * Gy * Gz


def _global_node(mesh, k, e, ix, iy, iz):
    Gx, Gy, _ = grid_dims(mesh, k)
    i, j, l = mesh.cell_ijk(e)
    return ((l * k + iz) * Gy + (j * k + iy)) * Gx + (i * k + ix)


def injection(mesh, k, ncomp):
    """P (N_DG x N_CG): DG coefficient of (cell, component, local node) = global value."""
    n = k + 1
    n3 = n ** 3
    Ng = n_cg(mesh, k, 1)
    rows, cols = [], []
    for e in range(mesh.n_cells):
        for c in range(ncomp):
            for iz in range(n):
                for iy in range(n):
                    for ix in range(n):
                        rows.append((e * ncomp + c) * n3 + (iz * n + iy) * n + ix)
                        cols.append(c * Ng + _global_node(mesh, k, e, ix, iy, iz))
    return sp.coo_matrix((np.ones(len(rows)), (rows, cols)),
                         shape=(mesh.n_cells * ncomp * n3, ncomp * Ng)).tocsr()


def pick(mesh, k, ncomp):
    """R (N_CG x N_DG): each global node from the lowest-index cell that holds it."""
    n = k + 1
    n3 = n ** 3
    Gx, Gy, Gz = grid_dims(mesh, k)
    Ng = Gx * Gy * Gz
    nx, ny, _ = mesh.n_cells_dir

    def cell_local(g):
        if g > 0 and g % k == 0:
            return g // k - 1, k
        return g // k, g % k

    rows, cols = [], []
    for gz in range(Gz):
        cz, iz = cell_local(gz)
        for gy in range(Gy):
            cy, iy = cell_local(gy)
            for gx in range(Gx):
                cx, ix = cell_local(gx)
                e = (cz * ny + cy) * nx + cx
                for c in range(ncomp):
                    rows.append(c * Ng + (gz * Gy + gy) * Gx + gx)
                    cols.append((e * ncomp + c) * n3 + (iz * n + iy) * n + ix)
    return sp.coo_matrix((np.ones(len(rows)), (rows, cols)),
                         shape=(ncomp * Ng, mesh.n_cells * ncomp * n3)).tocsr()


def cph_levels(levels, dg_mats, ncomp):
    """cph level matrices and prolongations for the DG sequence ``levels`` [(mesh, k), ...]
    (fine to coarse, as oracle.multigrid.level_sequence) with DG matrices ``dg_mats``.

    Returns (mats, prolongations): mats = [A_0, P_0^T A_0 P_0, P_1^T A_1 P_1, ...],
    prolongations[l] maps level l+1 to level l."""
    Ps = [injection(m, k, ncomp) for m, k in levels]
    Rs = [pick(m, k, ncomp) for m, k in levels]
    mats = [dg_mats[0]] + [(P.T @ A @ P).tocsr() for P, A in zip(Ps, dg_mats)]
    pro = [Ps[0]]
    for j in range(len(levels) - 1):
        (mf, kf), (mc, kc) = levels[j], levels[j + 1]
        if mf.n_cells == mc.n_cells:
            Pdg = omg.prolongation_p(mf, kf, kc, ncomp)
        else:
            Pdg = omg.prolongation_h(mf, mc, kf, ncomp)
        pro.append((Rs[j] @ Pdg @ Ps[j + 1]).tocsr())
    return mats, pro


def global_nodes(mesh, k):
    """(N_g, 3) coordinates of the global Gauss-Lobatto grid of a box mesh."""
    from . import quadrature
    x, _ = quadrature.gauss_lobatto(k + 1)
    coords = []
    for d, nc in enumerate(mesh.n_cells_dir):
        h = mesh.h[d]
        pts = [(c + x[i]) * h for c in range(nc) for i in range(k)] + [nc * h]
        coords.append(np.array(pts))
    Z, Y, X = np.meshgrid(coords[2], coords[1], coords[0], indexing='ij')
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
