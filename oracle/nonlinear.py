"""Picard iteration of the viscosity with Aitken relaxation (oracle, test infrastructure).

Sec. 5.4 (projection solver, Alg. 1 "projection solver with optionally
nonlinear viscous step"): with the convective term explicit (alpha_c = 0) the
viscous step, Eq. (viscous_step_weak), is nonlinear only through the
viscosity. The paper linearises it with a Picard update of the viscosity,
Eq. (viscosity_pointwise),
    nu^{n+1,k+1} = eta(gamma_dot(eps(u^{n+1,k}))),
solves the linear viscous step with that viscosity, and repeats until the
norm of the full nonlinear residual of the viscous step
    r^{visc,k} = b - (gamma_0/dt M + A(nu(u^k))) u^k
has dropped below eps_rel ||r^{visc,0}|| or below eps_abs. The iterate update
is accelerated with Aitken's adaptive relaxation (Irons and Tuck 1969), with
the relaxation factor computed from the full nonlinear residuals rather than
from the fixed-point increments (Sec. 5.4, the sentence after the stopping
rule).

READINGS (the paper prints no formulas for these):
* Aitken factor (Irons-Tuck form on residual vectors):
      omega_k = -omega_{k-1} r_{k-1} . (r_k - r_{k-1}) / ||r_k - r_{k-1}||^2,
  applied as u^{k+1} = u^k + omega_k (u_tilde^{k+1} - u^k) where u_tilde^{k+1}
  solves the viscous step linearised at u^k. omega_0 = omega_init (1: the
  first step is a plain Picard step). No clipping; a zero denominator keeps
  the previous factor.
* Stopping rule: the prose says convergence is reached "as soon as" EITHER the
  relative OR the absolute criterion holds, while the printed loop condition
  reads as if both had to hold; the prose is taken.
* The residual of the final iterate is evaluated with the viscosity updated
  from that iterate, so the returned viscosity is nu(u^final).
* Each linear solve starts from the current iterate u^k; its initial residual
  is then exactly r^{visc,k}, and it is solved to max(lin_rtol ||r^k||, lin_atol).

This module writes the loop once for any nonlinear residual (``picard_aitken``)
and once for the SIPG viscous step (``viscous_step_picard``), whose linear
solves are exact (sparse LU of the assembled matrix) so that the iterates are
those of the method without a solver tolerance in the way.

Pins (tests/test_oracle_nonlinear.py): on a linear residual with an inexact
(scaled) solve, Aitken relaxation lands on the fixed point at the second update
(closed form: omega_1 = 1/(alpha beta)); a constant viscosity converges after
one solve to the linear solution; the converged Carreau-Yasuda viscous step
agrees with an independent library root finder (scipy) on a tiny mesh; the
stopping rule stops as soon as either criterion holds.
"""
import numpy as np
import scipy.sparse.linalg as spla


def picard_aitken(update, operator, solve, b, u0, rtol=1e-8, atol=0.0, maxit=50, aitken=True,
                  omega_init=1.0, lin_rtol=1e-12, lin_atol=0.0):
    """Generic loop of Alg. 1 (viscous part).

    update(u)                -> linearisation state (the viscosity) evaluated at u
    operator(state, x)       -> (gamma_0/dt M + A(state)) x
    solve(state, b, x0, tol) -> solution of operator(state, .) = b (absolute tolerance tol)

    Returns a dict: u, state (at u), iterations, residuals ||r^k|| for k = 0..iterations,
    omegas (one per update), converged."""
    b = np.asarray(b, dtype=np.float64)
    u = np.array(u0, dtype=np.float64)
    state = update(u)
    r = b - operator(state, u)
    res = [float(np.linalg.norm(r))]
    omegas = []
    omega = float(omega_init)
    r_prev = None
    k = 0

    def converged():
        return res[-1] <= rtol * res[0] or res[-1] <= atol

    while k < maxit and not converged():
        u_tilde = solve(state, b, u, max(lin_rtol * res[-1], lin_atol))
        if aitken and r_prev is not None:
            dr = r - r_prev
            den = float(np.dot(dr, dr))
            if den > 0.0:
                omega = -omega * float(np.dot(r_prev, dr)) / den
        elif not aitken:
            omega = 1.0
        omegas.append(omega)
        u = u + omega * (u_tilde - u)
        r_prev = r
        state = update(u)
        r = b - operator(state, u)
        res.append(float(np.linalg.norm(r)))
        k += 1
    return {'u': u, 'state': state, 'iterations': k, 'residuals': res, 'omegas': omegas,
            'converged': converged()}


def viscous_step_picard(sipg, rheology, b, u0, mass, **kw):
    """Viscous step (gamma_0/dt) M u + A(nu(u)) u = b with the Picard/Aitken loop.

    sipg: oracle.sipg.SIPG with ncomp = 3; rheology: a velocity-dependent law
    (Carreau-Yasuda) or any other (then one solve converges); mass = gamma_0/dt."""
    def update(u):
        return sipg.viscosity_at_points(rheology, u)

    def operator(state, x):
        return sipg.apply(x, state[0], state[1], mass=mass)

    def solve(state, rhs, x0, tol):
        A = sipg.assemble(state[0], state[1], mass=mass).tocsc()
        return spla.spsolve(A, rhs)

    return picard_aitken(update, operator, solve, b, u0, **kw)
