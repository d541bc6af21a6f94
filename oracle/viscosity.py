"""Viscosity laws (oracle, test infrastructure).

* Shear rate, Sec. 2: gamma_dot = sqrt(2 eps(u) : eps(u)), eps = sym grad u.
* Generalized-Newtonian law, Eq. (viscosity_general):
      eta(gdot) = eta_inf + (eta_0 - eta_inf) * (kappa + (lambda*gdot)^a)^((b-1)/a)
  (Carreau-Yasuda for kappa = 1).
* Analytic field nu(x) = 1 + 9 sin^2(pi x) sin^2(pi y) sin^2(pi z) (contrast 10).
* Sphere ("sinker") field: nu_max inside any sphere |x - c_i| <= r, nu_matrix
  elsewhere; a point on a sphere surface counts as inside.
Pinned in tests/test_oracle_viscosity.py by the law's limits (gdot = 0 gives
eta_0, the excess over eta_inf decays like (lambda gdot)^(b-1), eta_0 = eta_inf
gives a constant), the closed-form value at lambda gdot = 1 (kappa = 1, a = 2,
b = 1/2: eta_inf + (eta_0 - eta_inf) 2^(-1/4)), the power law at kappa = 0 for
any a, the shear rates of simple shear (|gamma|), planar extension (2|e|) and a
rigid rotation (0), frame invariance, closed-form values of the analytic field,
the sphere test on a surface point, and the law evaluated from interpolated
simple-shear and extension flows at every cell and face point.

A rheology is a dict: {'law': 'constant', 'nu': v}, {'law': 'analytic'},
{'law': 'sinker', 'centers': (m,3), 'radius': r, 'nu_max': a, 'nu_matrix': b,
'projection': 'cell' | 'pointwise'} (see ``sipg.SIPG.viscosity_at_points``)
or {'law': 'carreau', 'eta0', 'eta_inf', 'kappa', 'lam', 'a', 'b'}.
"""
import numpy as np


def strain_rate(grad):
    """eps = (G + G^T)/2 for G[..., k, l] = d u_k / d x_l."""
    return 0.5 * (grad + np.swapaxes(grad, -1, -2))


def shear_rate(grad):
    eps = strain_rate(grad)
    return np.sqrt(2.0 * np.sum(eps * eps, axis=(-2, -1)))


def generalized_newtonian(gdot, eta0, eta_inf, kappa, lam, a, b):
    return eta_inf + (eta0 - eta_inf) * (kappa + (lam * gdot) ** a) ** ((b - 1.0) / a)


def analytic_field(x):
    x = np.asarray(x, dtype=np.float64)
    s = np.sin(np.pi * x[..., 0]) ** 2 * np.sin(np.pi * x[..., 1]) ** 2 * np.sin(np.pi * x[..., 2]) ** 2
    return 1.0 + 9.0 * s


def sinker_field(x, centers, radius, nu_max, nu_matrix):
    x = np.asarray(x, dtype=np.float64)
    inside = np.zeros(x.shape[:-1], dtype=bool)
    for c in np.asarray(centers, dtype=np.float64):
        d2 = np.sum((x - c) ** 2, axis=-1)
        inside |= d2 <= radius * radius
    return np.where(inside, nu_max, nu_matrix)


def evaluate(rheology, x, grad=None):
    """nu at physical points x (..., 3); grad (..., 3, 3) for velocity laws."""
    law = rheology['law']
    if law == 'constant':
        return np.full(np.asarray(x).shape[:-1], float(rheology['nu']))
    if law == 'analytic':
        return analytic_field(x)
    if law == 'sinker':
        return sinker_field(x, rheology['centers'], rheology['radius'],
                            rheology['nu_max'], rheology['nu_matrix'])
    if law == 'carreau':
        if grad is None:
            raise ValueError("the Carreau-Yasuda law needs the velocity gradient")
        return generalized_newtonian(shear_rate(grad), rheology['eta0'], rheology['eta_inf'],
                                     rheology['kappa'], rheology['lam'], rheology['a'],
                                     rheology['b'])
    raise ValueError(f"unknown law {law!r}")
