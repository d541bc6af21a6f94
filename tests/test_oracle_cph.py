"""Pins for the oracle's continuous ("cph") multigrid levels (Sec. 5.4), no GPU.

* the injection P reproduces continuous polynomials exactly and R P = I;
* the composed continuous prolongation reproduces a continuous coarse
  polynomial on the finer continuous level exactly, for the degree step and
  the mesh step;
* the continuous Galerkin operators P^T A P are symmetric, definite with
  Dirichlet walls, and keep constants (Poisson) / rigid-body modes (viscous)
  in their kernel with all-Neumann walls;
* the continuous DoF count in closed form.
"""
import numpy as np
import pytest

from oracle import cph
from oracle import multigrid as omg
from oracle.mesh import BoxMesh
from oracle.sipg import SIPG


def _poly(x):
    return np.stack([x[:, 0] * x[:, 1] - 0.3 * x[:, 2], x[:, 1] ** 2 + x[:, 0], x[:, 2] * x[:, 0] + 1.0], axis=1)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_injection_exact_and_pick_inverse(k):
    mesh = BoxMesh(3, 2, 2, extent=(1.0, 0.8, 0.6))
    S = SIPG(mesh, k, 3)
    P, R = cph.injection(mesh, k, 3), cph.pick(mesh, k, 3)
    g = cph.global_nodes(mesh, k)
    vals = _poly(g)
    ucg = np.concatenate([vals[:, c] for c in range(3)])
    assert np.abs(P @ ucg - S.interpolate(_poly)).max() <= 1e-14
    assert np.abs((R @ P) - np.eye(P.shape[1])).max() == 0.0
    nx, ny, nz = mesh.n_cells_dir
    assert P.shape[1] == 3 * (nx * k + 1) * (ny * k + 1) * (nz * k + 1)


def test_composed_prolongation_exact():
    mesh = BoxMesh(4, 2, 2)
    levels = [(mesh, 3), (mesh, 2), (mesh, 1), (mesh.coarsen(), 1)]
    dg = [SIPG(m, k, 3).assemble(*SIPG(m, k, 3).viscosity_at_points({'law': 'constant', 'nu': 1.0}))
          for m, k in levels]
    mats, pro = cph.cph_levels(levels, dg, 3)
    # a bilinear continuous field is represented exactly on every level
    f = lambda x: np.stack([x[:, 0] * x[:, 1], x[:, 2] + 0.5 * x[:, 0], x[:, 1] * x[:, 2]], axis=1)
    cg = []
    for m, k in levels:
        v = f(cph.global_nodes(m, k))
        cg.append(np.concatenate([v[:, c] for c in range(3)]))
    for j in range(len(levels) - 1):
        # pro[j + 1] maps continuous level j+1 to continuous level j
        assert np.abs(pro[j + 1] @ cg[j + 1] - cg[j]).max() <= 1e-13
    assert np.abs(pro[0] @ cg[0] - SIPG(mesh, 3, 3).interpolate(f)).max() <= 1e-13


def test_continuous_operators():
    mesh = BoxMesh(2, 2, 2)
    k = 2
    S = SIPG(mesh, k, 3)
    A = S.assemble(*S.viscosity_at_points({'law': 'analytic'})).toarray()
    P = cph.injection(mesh, k, 3).toarray()
    Acg = P.T @ A @ P
    assert np.abs(Acg - Acg.T).max() <= 1e-13 * np.abs(Acg).max()
    assert np.linalg.eigvalsh(Acg).min() > 0
    meshn = BoxMesh(2, 2, 2, bc=('N',) * 6)
    Sn = SIPG(meshn, k, 3)
    An = Sn.assemble(*Sn.viscosity_at_points({'law': 'analytic'})).toarray()
    Pn = cph.injection(meshn, k, 3).toarray()
    Acgn = Pn.T @ An @ Pn
    g = cph.global_nodes(meshn, k)
    for b in np.eye(3):
        r = np.cross(b, g)
        v = np.concatenate([r[:, c] for c in range(3)])
        assert np.abs(Acgn @ v).max() <= 1e-12 * np.abs(Acgn).max()
    Sp = SIPG(meshn, 2, 1)
    Ap = Sp.assemble().toarray()
    Pp = cph.injection(meshn, 2, 1).toarray()
    assert np.abs((Pp.T @ Ap @ Pp) @ np.ones(Pp.shape[1])).max() <= 1e-12 * np.abs(Ap).max()


def test_cph_vcycle_reduces_the_error():
    mesh = BoxMesh(4, 4, 4)
    levels = omg.level_sequence(mesh, 2, 3, coarse_threshold=300)
    dg = []
    for m, k in levels:
        S = SIPG(m, k, 3)
        dg.append(S.assemble(*S.viscosity_at_points({'law': 'analytic'})))
    mats, pro = cph.cph_levels(levels, dg, 3)
    lmax = [1.2 * omg.lanczos_lmax(A, omg.inverse_diagonal(A), np.ones(A.shape[0]), 15) for A in mats[:-1]]
    V = omg.VCycle(mats, pro, 3, lmax)
    A = mats[0]
    x = np.random.default_rng(0).standard_normal(A.shape[0])
    b = A @ x
    e1 = x - V(b)
    assert np.linalg.norm(e1) <= 0.5 * np.linalg.norm(x)
