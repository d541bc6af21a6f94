"""Krylov and direct solvers on assembled matrices (oracle, test infrastructure).

Sec. 5.4: the viscous and pressure steps are solved with the conjugate gradient
method. The oracle uses the textbook preconditioned CG (Hestenes-Stiefel, as in
Saad 2003, Alg. 9.1) with an optional preconditioner callable, and a dense
Cholesky solve for small systems. A preconditioner does not change the discrete
solution, so the oracle's reference solutions come from Jacobi-PCG to a tight
tolerance or from the dense factorization.
"""
import numpy as np
import scipy.linalg as sla


def _as_op(A):
    return A if callable(A) else (lambda v: A @ v)


def pcg(A, b, x0=None, precond=None, rtol=1e-10, atol=0.0, maxit=10000, project=None):
    """Preconditioned CG. Returns (x, iterations, relative residual history).

    project: optional map applied to residuals and search directions (used to
    keep iterates in the complement of a null space, e.g. constants)."""
    op = _as_op(A)
    M = precond if precond is not None else (lambda r: r.copy())
    P = project if project is not None else (lambda v: v)
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = P(b - op(x))
    bnorm = np.linalg.norm(P(b))
    hist = [np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0]
    if bnorm == 0.0:
        return x, 0, hist
    z = P(M(r))
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        if np.linalg.norm(r) <= max(rtol * bnorm, atol):
            break
        Ap = op(p)
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        r = P(r)
        it += 1
        hist.append(np.linalg.norm(r) / bnorm)
        z = P(M(r))
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist


def jacobi_pcg(A, b, **kw):
    d = A.diagonal()
    return pcg(A, b, precond=lambda r: r / d, **kw)


def cholesky_solve(A, b):
    """Dense SPD solve by Cholesky factorization."""
    A = np.asarray(A.toarray() if hasattr(A, 'toarray') else A, dtype=np.float64)
    c = sla.cho_factor(A, lower=True)
    return sla.cho_solve(c, b)
