"""Pins for the oracle's Picard/Aitken loop of the viscous step (Sec. 5.4, Alg. 1).

* closed form: for a linear residual r(u) = b - alpha u and an inexact solve
  that returns u + beta r(u), Aitken's factor after the first update is
  1/(alpha beta) and the second update lands on the fixed point b/alpha;
  plain Picard contracts by exactly |1 - alpha beta| per update;
* a constant viscosity converges after one update to the linear solution;
* the Carreau-Yasuda viscous step converged by the loop satisfies the
  nonlinear equations found independently by scipy's root finder;
* the stopping rule stops as soon as either criterion holds.
"""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse.linalg as spla

from oracle import mass, nonlinear
from oracle.mesh import BoxMesh
from oracle.sipg import SIPG
from paper_2506_14424_gb300 import inputs


def _linear_problem(alpha, beta):
    def update(u):
        return None

    def operator(state, x):
        return alpha * x

    def solve(state, b, x0, tol):
        return x0 + beta * (b - alpha * x0)

    return update, operator, solve


@pytest.mark.parametrize("alpha,beta", [(2.0, 0.3), (0.5, 3.0), (4.0, 0.1)])
def test_aitken_closed_form(alpha, beta):
    b = np.random.default_rng(1).standard_normal(5)
    u0 = np.random.default_rng(2).standard_normal(5)
    out = nonlinear.picard_aitken(*_linear_problem(alpha, beta), b, u0, rtol=1e-13, maxit=2, aitken=True)
    assert out['omegas'][0] == 1.0
    assert abs(out['omegas'][1] - 1.0 / (alpha * beta)) <= 1e-12 / (alpha * beta)
    assert np.abs(out['u'] - b / alpha).max() <= 1e-12 * np.abs(b / alpha).max()


@pytest.mark.parametrize("alpha,beta", [(2.0, 0.3), (0.5, 3.0)])
def test_plain_picard_contraction(alpha, beta):
    b = np.random.default_rng(3).standard_normal(4)
    out = nonlinear.picard_aitken(*_linear_problem(alpha, beta), b, np.zeros(4), rtol=0.0, maxit=6,
                                  aitken=False)
    res = np.array(out['residuals'])
    assert np.allclose(res[1:] / res[:-1], abs(1.0 - alpha * beta), rtol=1e-10)
    assert out['omegas'] == [1.0] * 6


def _problem(dims=(2, 1, 1), k=2, m=10.0, amp=1.0):
    S = SIPG(BoxMesh(*dims), k, 3)
    modes = inputs.fourier_modes(3)
    uh = S.interpolate(lambda x: amp * inputs.fourier_field(x, modes))
    return S, uh, mass.apply_mass(S, uh, m), m


def test_constant_viscosity_one_update():
    S, uh, b, m = _problem()
    rh = {'law': 'constant', 'nu': 0.7}
    out = nonlinear.viscous_step_picard(S, rh, b, uh, m, rtol=1e-12, maxit=5)
    assert out['iterations'] == 1 and out['converged']
    nc, nf = S.viscosity_at_points(rh)
    ref = spla.spsolve(S.assemble(nc, nf, mass=m).tocsc(), b)
    assert np.abs(out['u'] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_carreau_matches_library_root():
    S, uh, b, m = _problem()
    rh = inputs.carreau_blood_like()
    out = nonlinear.viscous_step_picard(S, rh, b, uh, m, rtol=1e-13, maxit=60)
    assert out['converged']

    def R(u):
        nc, nf = S.viscosity_at_points(rh, u)
        return b - S.apply(u, nc, nf, mass=m)

    sol = so.root(R, uh, method='hybr', options={'xtol': 1e-13})
    assert sol.success
    assert np.abs(R(sol.x)).max() <= 1e-9 * np.abs(b).max()
    assert np.abs(out['u'] - sol.x).max() <= 1e-9 * np.abs(sol.x).max()


def test_stopping_rule_either_criterion():
    S, uh, b, m = _problem()
    rh = inputs.carreau_blood_like()
    first = nonlinear.viscous_step_picard(S, rh, b, uh, m, rtol=0.0, maxit=0)
    r0 = first['residuals'][0]
    # the absolute criterion alone stops the loop although the relative one does not hold
    out = nonlinear.viscous_step_picard(S, rh, b, uh, m, rtol=1e-30, atol=2.0 * r0, maxit=10)
    assert out['iterations'] == 0 and out['converged']
    # and the relative one alone stops it
    out = nonlinear.viscous_step_picard(S, rh, b, uh, m, rtol=0.5, atol=0.0, maxit=10)
    assert out['iterations'] == 1 and out['residuals'][1] <= 0.5 * r0
