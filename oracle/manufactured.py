"""Manufactured solutions and load vectors (oracle, test infrastructure).

Sec. 7.1 verifies optimal spatial convergence (order k+1 in L2) with a
manufactured solution. Here the same check is run on the steady viscous
operator alone: -div(2 nu eps(u)) = f in the unit cube, u = 0 on the walls.

Velocity case: u = s(x) c, s = sin(pi x) sin(pi y) sin(pi z), c = (1, -1, 2),
with the analytic viscosity nu = 1 + 9 sin^2(pi x) sin^2(pi y) sin^2(pi z)
(= 1 + 9 s^2). Differentiating by hand:
    f_i = -2 sum_j eps_ij d_j nu - nu (c_i lap s + sum_j c_j d_i d_j s),
    eps_ij = (c_i d_j s + c_j d_i s) / 2,  d_j nu = 18 s d_j s.
Pressure case: p = cos(pi x) cos(pi y) cos(pi z), -lap p = 3 pi^2 p, zero normal
derivative on the walls and zero mean.
Pinned in tests against central finite differences of the flux 2 nu eps(u).
"""
import numpy as np

from . import basis, quadrature

C_VEC = np.array([1.0, -1.0, 2.0])


def s_and_derivs(x):
    x = np.asarray(x, dtype=np.float64)
    S = np.sin(np.pi * x)
    Cc = np.cos(np.pi * x)
    s = S[..., 0] * S[..., 1] * S[..., 2]
    grad = np.stack([np.pi * Cc[..., 0] * S[..., 1] * S[..., 2],
                     np.pi * S[..., 0] * Cc[..., 1] * S[..., 2],
                     np.pi * S[..., 0] * S[..., 1] * Cc[..., 2]], axis=-1)
    hess = np.zeros(x.shape[:-1] + (3, 3))
    for i in range(3):
        for j in range(3):
            if i == j:
                hess[..., i, j] = -np.pi ** 2 * s
            else:
                m = 3 - i - j
                hess[..., i, j] = np.pi ** 2 * Cc[..., i] * Cc[..., j] * S[..., m]
    return s, grad, hess


def velocity_exact(x):
    s, _, _ = s_and_derivs(x)
    return s[..., None] * C_VEC


def velocity_force(x):
    s, g, H = s_and_derivs(x)
    nu = 1.0 + 9.0 * s * s
    dnu = 18.0 * s[..., None] * g
    eps = 0.5 * (C_VEC[:, None] * g[..., None, :] + g[..., :, None] * C_VEC[None, :])
    lap = np.trace(H, axis1=-2, axis2=-1)
    f = -2.0 * np.einsum('...ij,...j->...i', eps, dnu) \
        - nu[..., None] * (C_VEC * lap[..., None] + np.einsum('...ij,j->...i', H, C_VEC))
    return f


def pressure_exact(x):
    x = np.asarray(x, dtype=np.float64)
    return np.cos(np.pi * x[..., 0]) * np.cos(np.pi * x[..., 1]) * np.cos(np.pi * x[..., 2])


def pressure_force(x):
    return 3.0 * np.pi ** 2 * pressure_exact(x)


def _fine_rule(disc, extra):
    nq = disc.n + extra
    g, w = quadrature.gauss_legendre(nq)
    qz, qy, qx = np.meshgrid(np.arange(nq), np.arange(nq), np.arange(nq), indexing='ij')
    xi = np.stack([g[qx.ravel()], g[qy.ravel()], g[qz.ravel()]], axis=1)
    W = w[qx.ravel()] * w[qy.ravel()] * w[qz.ravel()]
    phi, _ = basis.tensor_basis(disc.nodes, xi)
    return xi, W, phi


def load_vector(disc, force, extra=3):
    """b[(e, c, i)] = integral of phi_i f_c over cell e (over-integrated)."""
    xi, W, phi = _fine_rule(disc, extra)
    detJ = disc.mesh.volume()
    out = np.zeros((disc.mesh.n_cells, disc.ncomp, disc.n ** 3))
    for e in range(disc.mesh.n_cells):
        pts = disc.mesh.origin(e) + xi * disc.mesh.h
        f = np.asarray(force(pts)).reshape(len(W), disc.ncomp)
        out[e] = np.einsum('q,qi,qc->ci', W * detJ, phi, f)
    return out.reshape(-1)


def l2_error(disc, uh, exact, extra=3):
    xi, W, phi = _fine_rule(disc, extra)
    detJ = disc.mesh.volume()
    U = np.asarray(uh).reshape(disc.mesh.n_cells, disc.ncomp, disc.n ** 3)
    err2 = 0.0
    for e in range(disc.mesh.n_cells):
        pts = disc.mesh.origin(e) + xi * disc.mesh.h
        ue = np.asarray(exact(pts)).reshape(len(W), disc.ncomp)
        uh_q = np.einsum('qi,ci->qc', phi, U[e])
        err2 += np.sum(W * detJ * np.sum((uh_q - ue) ** 2, axis=1))
    return np.sqrt(err2)
