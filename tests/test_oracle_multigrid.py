"""Pins for the oracle's multigrid pieces and CG (no GPU).

* prolongation (embedding) reproduces coarse polynomials exactly at the fine
  nodes, for p- and h-transfers; restriction is its transpose;
* downward interpolation of the linearization velocity is exact on functions
  the coarse space holds;
* the Chebyshev-Jacobi smoother's error propagation equals the closed-form
  scaled Chebyshev polynomial on eigenvectors of D^-1 A;
* the Lanczos estimate is a lower bound of the largest eigenvalue and close to it;
* PCG reaches the dense Cholesky solution.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import multigrid as mg, solvers
from oracle.mesh import BoxMesh
from oracle.sipg import SIPG


def _poly(p):
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    return np.stack([1 + x - 2 * y + 0.5 * z + x * y * z, x * z - y, 2 - z + x * y], axis=1)


@pytest.mark.parametrize("kf,kc", [(2, 1), (3, 2), (4, 2), (5, 2)])
def test_p_prolongation_exact(kf, kc):
    mesh = BoxMesh(2, 1, 2, extent=(1.0, 0.5, 1.5))
    Sf, Sc = SIPG(mesh, kf, 3), SIPG(mesh, kc, 3)
    P = mg.prolongation_p(mesh, kf, kc, 3)
    assert np.abs(P @ Sc.interpolate(_poly) - Sf.interpolate(_poly)).max() < 1e-13
    # downward interpolation recovers the coarse interpolant of a coarse-space function
    assert np.abs(mg.interpolate_down_p(Sf.interpolate(_poly), mesh, kf, kc, 3)
                  - Sc.interpolate(_poly)).max() < 1e-13


@pytest.mark.parametrize("k", [1, 2])
def test_h_prolongation_exact(k):
    fine = BoxMesh(4, 2, 2)
    coarse = fine.coarsen()
    Sf, Sc = SIPG(fine, k, 3), SIPG(coarse, k, 3)
    P = mg.prolongation_h(fine, coarse, k, 3)
    assert np.abs(P @ Sc.interpolate(_poly) - Sf.interpolate(_poly)).max() < 1e-13
    assert np.abs(mg.interpolate_down_h(Sf.interpolate(_poly), fine, coarse, k, 3)
                  - Sc.interpolate(_poly)).max() < 1e-13


def test_level_sequence_16cubed_k4_shape():
    levels = mg.level_sequence(BoxMesh(16, 16, 16), 4, 3)
    desc = [(m.n_cells_dir[0], k) for m, k in levels]
    assert desc == [(16, 4), (16, 2), (16, 1), (8, 1), (4, 1)]
    assert levels[-1][0].n_cells * 3 * 8 == 1536


def test_chebyshev_closed_form_on_eigenvectors():
    S = SIPG(BoxMesh(2, 2, 1), 2, 3)
    A = S.assemble(*S.viscosity_at_points({'law': 'analytic'})).toarray()
    dinv = 1.0 / np.diag(A)
    # eigenpairs of D^-1 A via the symmetric form D^-1/2 A D^-1/2
    s = np.sqrt(dinv)
    lam, Q = np.linalg.eigh(s[:, None] * A * s[None, :])
    lmax = 1.2 * lam[-1]
    lmin = lmax / 20.0
    for idx in [0, len(lam) // 3, len(lam) - 1]:
        v = s * Q[:, idx]          # eigenvector of D^-1 A
        b = np.zeros_like(v)
        # smoothing A x = 0 from x0 = v: the error after the smoother is p(lam) v
        x = mg.chebyshev(A, dinv, b, v, 3, lmin, lmax)
        expect = mg.chebyshev_error_polynomial(lam[idx], 3, lmin, lmax)
        assert np.abs(x - expect * v).max() < 1e-10 * np.abs(v).max()


def test_lanczos_estimate_bounds():
    S = SIPG(BoxMesh(2, 2, 2), 2, 3)
    A = S.assemble(*S.viscosity_at_points({'law': 'analytic'})).toarray()
    dinv = 1.0 / np.diag(A)
    s = np.sqrt(dinv)
    exact = np.linalg.eigvalsh(s[:, None] * A * s[None, :])[-1]
    est = mg.lanczos_lmax(A, dinv, np.random.default_rng(0).uniform(-1, 1, A.shape[0]), 15)
    assert est <= exact * (1 + 1e-12) and est > 0.9 * exact


def test_pcg_matches_cholesky():
    S = SIPG(BoxMesh(2, 2, 2), 2, 3)
    A = S.assemble(*S.viscosity_at_points({'law': 'analytic'}))
    b = np.random.default_rng(1).uniform(-1, 1, A.shape[0])
    x_ref = solvers.cholesky_solve(A, b)
    x, it, hist = solvers.jacobi_pcg(A, b, rtol=1e-13)
    assert np.abs(x - x_ref).max() < 1e-10 * np.abs(x_ref).max()
    assert hist[-1] <= 1e-13


def test_vcycle_preconditioned_cg_converges_fast():
    mesh = BoxMesh(4, 4, 4)
    levels = mg.level_sequence(mesh, 2, 3, coarse_threshold=700)
    mats, Ps = [], []
    for l, (m, k) in enumerate(levels):
        S = SIPG(m, k, 3)
        mats.append(S.assemble(*S.viscosity_at_points({'law': 'analytic'})))
        if l > 0:
            pm, pk = levels[l - 1]
            Ps.append(mg.prolongation_p(m, pk, k, 3) if pm is m else mg.prolongation_h(pm, m, k, 3))
    lmax = []
    for A in mats[:-1]:
        d = 1.0 / A.diagonal()
        lmax.append(1.2 * mg.lanczos_lmax(A, d, np.random.default_rng(0).uniform(-1, 1, A.shape[0]), 15))
    V = mg.VCycle(mats, Ps, 3, lmax)
    b = np.random.default_rng(3).uniform(-1, 1, mats[0].shape[0])
    x, it, hist = solvers.pcg(mats[0], b, precond=V, rtol=1e-8)
    assert hist[-1] <= 1e-8 and it <= 25, it
    x_ref = solvers.cholesky_solve(mats[0], b)
    assert np.abs(x - x_ref).max() <= 1e-6 * np.abs(x_ref).max()


def _sinker_vcycle_iterations(levels_visc):
    mats, Ps = [], []
    for l, ((m, k), nu) in enumerate(levels_visc):
        S = SIPG(m, k, 3)
        mats.append(S.assemble(*nu))
        if l > 0:
            pm, pk = levels_visc[l - 1][0]
            Ps.append(mg.prolongation_p(m, pk, k, 3) if pm.n_cells == m.n_cells else mg.prolongation_h(pm, m, k, 3))
    lmax = [1.2 * mg.lanczos_lmax(A, 1.0 / A.diagonal(), np.random.default_rng(0).uniform(-1, 1, A.shape[0]), 15)
            for A in mats[:-1]]
    V = mg.VCycle(mats, Ps, 3, lmax)
    b = mats[0] @ np.random.default_rng(1).uniform(-1, 1, mats[0].shape[0])
    return solvers.pcg(mats[0], b, precond=V, rtol=1e-8, maxit=150)[1]


def test_transferred_sinker_viscosity_keeps_vcycle_robust():
    """Finding behind the viscosity-transfer reading: at contrast 1e4 the V-cycle
    with transferred cell values converges in a few dozen CG iterations, with
    per-level re-evaluation it stalls."""
    from paper_2506_14424_gb300 import inputs
    rheo = inputs.sinker(seed=2, count=8, radius=0.2, nu_max=1e4)
    levels = mg.level_sequence(BoxMesh(4, 4, 4), 2, 3, coarse_threshold=200)
    transferred = mg.level_viscosity(levels, rheo)
    reevaluated = [SIPG(m, k, 3).viscosity_at_points(rheo) for m, k in levels]
    assert _sinker_vcycle_iterations(list(zip(levels, transferred))) <= 35
    assert _sinker_vcycle_iterations(list(zip(levels, reevaluated))) >= 100
