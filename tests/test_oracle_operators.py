"""Pins for the oracle's SIPG operators against what the paper and mathematics fix (no GPU).

* symmetry of the symmetric interior penalty forms (Sec. 5.1, 5.2);
* null spaces: rigid-body modes for the all-Neumann viscous operator (this pins
  the symmetric gradient eps(u) of Sec. 2) and constants for the all-Neumann
  Poisson operator (Sec. 3.2, pure-Dirichlet velocity => pressure up to a constant);
* positive definiteness with Dirichlet walls for viscosity contrasts 1..1e6;
* brute-force quadrature: k+1 Gauss points are exact for constant nu, so k+4
  points give the same matrix;
* Galerkin consistency: for a Q_2 field vanishing on the walls the discrete
  operator reproduces the exact load;
* DoF counting of the cavity workload (Sec. 7.3: 32^3 cells, k_u = 4, 14.4e6 DoFs);
* optimal order k+1 in L2 (Sec. 7.1, Fig. convergence_space).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import manufactured, solvers
from oracle.mesh import BoxMesh
from oracle.sipg import SIPG
from paper_2506_14424_gb300 import inputs


def _viscous(mesh, k, rheo={'law': 'analytic'}, **kw):
    S = SIPG(mesh, k, 3, **kw)
    nc, nf = S.viscosity_at_points(rheo)
    return S, S.assemble(nc, nf).toarray()


@pytest.mark.parametrize("dims,k", [((2, 2, 2), 1), ((3, 2, 1), 2), ((1, 2, 2), 3)])
def test_viscous_symmetric(dims, k):
    _, A = _viscous(BoxMesh(*dims), k)
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()


@pytest.mark.parametrize("dims,k", [((2, 2, 2), 2), ((3, 1, 2), 3)])
def test_poisson_symmetric(dims, k):
    P = SIPG(BoxMesh(*dims), k, 1)
    A = P.assemble().toarray()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()


def _rigid(i):
    def f(p):
        x = p - 0.5
        if i < 3:
            v = np.zeros_like(p)
            v[:, i] = 1.0
            return v
        b = np.zeros(3)
        b[i - 3] = 1.0
        return np.cross(b, x)
    return f


@pytest.mark.parametrize("k", [1, 2, 3])
def test_viscous_neumann_rigid_body_null_space(k):
    S, A = _viscous(BoxMesh(2, 2, 1, bc=('N',) * 6), k)
    scale = np.abs(A).max()
    for i in range(6):
        r = S.interpolate(_rigid(i))
        assert np.abs(A @ r).max() <= 1e-13 * scale * np.abs(r).max()
    # and nothing else: exactly six zero eigenvalues
    ev = np.linalg.eigvalsh(A)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 6


def test_viscous_dirichlet_kills_rigid_modes():
    S, A = _viscous(BoxMesh(2, 2, 2), 2)
    for i in range(6):
        r = S.interpolate(_rigid(i))
        assert np.abs(A @ r).max() > 1e-3


@pytest.mark.parametrize("k", [1, 2, 3])
def test_poisson_neumann_constant_null_space(k):
    P = SIPG(BoxMesh(2, 3, 2, bc=('N',) * 6), k, 1)
    A = P.assemble().toarray()
    one = np.ones(A.shape[0])
    assert np.abs(A @ one).max() <= 1e-13 * np.abs(A).max()
    ev = np.linalg.eigvalsh(A)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 1


@pytest.mark.parametrize("contrast", [1.0, 1e2, 1e4, 1e6])
def test_viscous_dirichlet_spd_sinker(contrast):
    rheo = inputs.sinker(seed=2, count=8, radius=0.3, nu_max=contrast)
    _, A = _viscous(BoxMesh(2, 2, 2), 2, rheo)
    sla.cholesky(A, lower=True)            # raises if not SPD
    ev = np.linalg.eigvalsh(A)
    assert ev[0] > 0.0


@pytest.mark.parametrize("mode", ["max", "arith"])
def test_viscous_spd_face_modes_contrast_1e6(mode):
    rheo = inputs.sinker(seed=2, count=8, radius=0.3, nu_max=1e6)
    _, A = _viscous(BoxMesh(2, 2, 2), 2, rheo, face_nu=mode)
    assert np.linalg.eigvalsh(A)[0] > 0.0


def test_viscous_spd_sinker_cfg_like_mesh():
    """4^3 cells, radius-0.1 spheres cutting through cells, contrast 1e6."""
    rheo = inputs.sinker(seed=2, count=8, radius=0.1, nu_max=1e6)
    _, A = _viscous(BoxMesh(4, 4, 4), 1, rheo)
    assert np.linalg.eigvalsh(A)[0] > 0.0


def test_pointwise_sinker_is_not_coercive():
    """The finding behind the cellwise projection: raw pointwise values lose SPD."""
    rheo = inputs.sinker(seed=2, count=8, radius=0.3, nu_max=1e4)
    rheo['projection'] = 'pointwise'
    _, A = _viscous(BoxMesh(2, 2, 2), 2, rheo)
    assert np.linalg.eigvalsh(A)[0] < 0.0


def test_poisson_dirichlet_spd():
    P = SIPG(BoxMesh(2, 2, 2), 2, 1)
    A = P.assemble().toarray()
    sla.cholesky(A, lower=True)


@pytest.mark.parametrize("dims,k", [((1, 1, 1), 2), ((2, 1, 1), 2), ((2, 1, 1), 3)])
def test_brute_force_quadrature_constant_nu(dims, k):
    mesh = BoxMesh(*dims, extent=(0.7, 0.4, 0.9))
    rheo = {'law': 'constant', 'nu': 0.37}
    S1 = SIPG(mesh, k, 3)
    S2 = SIPG(mesh, k, 3, n_quad=k + 4)
    A1 = S1.assemble(*S1.viscosity_at_points(rheo), mass=2.5).toarray()
    A2 = S2.assemble(*S2.viscosity_at_points(rheo), mass=2.5).toarray()
    assert np.abs(A1 - A2).max() <= 1e-13 * np.abs(A2).max()
    P1 = SIPG(mesh, k, 1).assemble().toarray()
    P2 = SIPG(mesh, k, 1, n_quad=k + 4).assemble().toarray()
    assert np.abs(P1 - P2).max() <= 1e-13 * np.abs(P2).max()


def _q_and_derivs(x):
    """q = x(1-x) y(1-y) z(1-z): value and Hessian, written out by hand."""
    a = x * (1 - x)
    da = 1 - 2 * x
    q = a[..., 0] * a[..., 1] * a[..., 2]
    H = np.zeros(x.shape[:-1] + (3, 3))
    for i in range(3):
        for j in range(3):
            if i == j:
                others = [m for m in range(3) if m != i]
                H[..., i, i] = -2.0 * a[..., others[0]] * a[..., others[1]]
            else:
                m = 3 - i - j
                H[..., i, j] = da[..., i] * da[..., j] * a[..., m]
    return q, H


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_viscous_galerkin_consistency_q2(comp):
    nu = 1.7
    mesh = BoxMesh(2, 2, 2)
    S = SIPG(mesh, 2, 3)
    A = S.assemble(*S.viscosity_at_points({'law': 'constant', 'nu': nu})).toarray()

    def u_exact(p):
        v = np.zeros_like(p)
        v[:, comp] = _q_and_derivs(p)[0]
        return v

    def force(p):
        _, H = _q_and_derivs(p)
        f = H[..., :, comp].copy()                      # grad (d_c q)
        f[..., comp] += np.trace(H, axis1=-2, axis2=-1)  # + lap q e_c
        return -nu * f

    u = S.interpolate(u_exact)
    b = manufactured.load_vector(S, force)
    assert np.abs(A @ u - b).max() <= 1e-13 * np.abs(b).max()


def test_poisson_galerkin_consistency_q2():
    """p = x^2 + 2 y^2 - z^2 in Q_2: A p = int phi (-lap p) + sum_walls int phi dp/dn."""
    mesh = BoxMesh(2, 2, 2, bc=('N',) * 6)
    P = SIPG(mesh, 2, 1)
    A = P.assemble().toarray()
    coef = np.array([1.0, 2.0, -1.0])
    p = P.interpolate(lambda x: (x ** 2 @ coef)[:, None])
    b = manufactured.load_vector(P, lambda x: np.full(x.shape[:-1] + (1,), -2.0 * coef.sum()))
    b = b.reshape(mesh.n_cells, -1)
    for e in range(mesh.n_cells):
        for f in range(6):
            if mesh.neighbor(e, f) is not None:
                continue
            d, s = divmod(f, 2)
            pts = P.face_points(e, f)
            dpdn = (2.0 * s - 1.0) * 2.0 * coef[d] * pts[:, d]
            b[e] += np.einsum('q,qi->i', P.face_w2 * mesh.face_area(d) * dpdn, P.face_phi[f])
    assert np.abs(A @ p - b.ravel()).max() <= 1e-13 * np.abs(b).max()


def test_dof_count_cavity_workload():
    """Sec. 7.3: 32^3 cells, k_u = 4, k_p = 3 -> 14.4e6 DoFs."""
    mesh = BoxMesh(32, 32, 32)
    cells = mesh.n_cells
    total = cells * 3 * (4 + 1) ** 3 + cells * (3 + 1) ** 3
    assert total == 14385152 and round(total / 1e5) / 10 == 14.4


def test_viscous_convergence_order_k_plus_1():
    errs = []
    for N in (2, 4, 8):
        S = SIPG(BoxMesh(N, N, N), 2, 3)
        A = S.assemble(*S.viscosity_at_points({'law': 'analytic'}))
        b = manufactured.load_vector(S, manufactured.velocity_force)
        x, _, _ = solvers.jacobi_pcg(A, b, rtol=1e-12)
        errs.append(manufactured.l2_error(S, x, manufactured.velocity_exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 2.8 and rates[-1] < 3.6, rates


def test_poisson_convergence_order_k_plus_1():
    errs = []
    for N in (2, 4, 8):
        P = SIPG(BoxMesh(N, N, N, bc=('N',) * 6), 1, 1)
        A = P.assemble()
        b = manufactured.load_vector(P, lambda x: manufactured.pressure_force(x)[..., None])
        proj = lambda v: v - v.mean()
        x, _, _ = solvers.pcg(A, b, rtol=1e-12, project=proj)
        # compare with the zero-mean exact pressure
        errs.append(manufactured.l2_error(P, x, lambda p: manufactured.pressure_exact(p)[..., None]))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 1.8, rates


def test_manufactured_force_matches_finite_differences():
    rng = np.random.default_rng(7)
    pts = rng.uniform(0.1, 0.9, size=(5, 3))
    h = 1e-5

    def flux(p):
        # 2 nu eps(u) from the closed forms of u and nu only
        s, g, _ = manufactured.s_and_derivs(p)
        nu = 1.0 + 9.0 * s * s
        G = manufactured.C_VEC[:, None] * g[..., None, :]
        return 2.0 * nu[..., None, None] * 0.5 * (G + np.swapaxes(G, -1, -2))

    div = np.zeros((5, 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        div += (flux(pts + e)[..., :, j] - flux(pts - e)[..., :, j]) / (2 * h)
    assert np.allclose(manufactured.velocity_force(pts), -div, rtol=1e-6, atol=1e-6)
