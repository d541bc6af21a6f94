"""Gauss-Legendre and Gauss-Lobatto rules on [0, 1] (oracle, test infrastructure).

The discrete spaces of Sec. 5 are tensor-product Q_k on hexahedra. Nodal
coefficients live on the k+1 Gauss-Lobatto points; integrals use k+1
Gauss-Legendre points per direction (the paper uses as many quadrature points
as support points, Sec. 5.1 "viscosity_pointwise" discussion).

Both rules are computed from their textbook definitions with Newton's method on
the Legendre polynomials P_m (three-term recurrence):
  * Gauss-Legendre with n points: the roots of P_n, weights
    2 / ((1 - x^2) P_n'(x)^2) on [-1, 1];
  * Gauss-Lobatto with n points: -1, +1 and the roots of P_{n-1}', weights
    2 / (n (n - 1) P_{n-1}(x)^2) on [-1, 1].
Pinned in tests by exactness on monomials (degree 2n-1, resp. 2n-3) and by the
closed-form low-order nodes.
"""
import numpy as np


def legendre(m, x):
    """Return (P_m(x), P_m'(x), P_m''(x)) by the Bonnet recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if m == 0:
        z = np.zeros_like(x)
        return p_prev, z, z
    p = x.copy()
    dp_prev = np.zeros_like(x)
    dp = np.ones_like(x)
    d2p_prev = np.zeros_like(x)
    d2p = np.zeros_like(x)
    for j in range(1, m):
        # (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1}, differentiated twice
        p_next = ((2 * j + 1) * x * p - j * p_prev) / (j + 1)
        dp_next = ((2 * j + 1) * (p + x * dp) - j * dp_prev) / (j + 1)
        d2p_next = ((2 * j + 1) * (2 * dp + x * d2p) - j * d2p_prev) / (j + 1)
        p_prev, p = p, p_next
        dp_prev, dp = dp, dp_next
        d2p_prev, d2p = d2p, d2p_next
    return p, dp, d2p


def _newton(f, x0, iters=100):
    x = np.array(x0, dtype=np.float64)
    for _ in range(iters):
        val, der = f(x)
        step = val / der
        x = x - step
        if np.max(np.abs(step)) < 1e-16:
            break
    return x


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0, 1]: (points ascending, weights)."""
    i = np.arange(1, n + 1)
    x0 = -np.cos(np.pi * (i - 0.25) / (n + 0.5))
    x = _newton(lambda t: legendre(n, t)[:2], x0)
    _, dp, _ = legendre(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss_lobatto(n):
    """n-point Gauss-Lobatto rule on [0, 1] (n >= 2): (points ascending, weights)."""
    if n < 2:
        raise ValueError("Gauss-Lobatto needs at least two points")
    m = n - 1
    x = np.empty(n)
    x[0], x[-1] = -1.0, 1.0
    if n > 2:
        j = np.arange(1, n - 1)
        x0 = -np.cos(np.pi * j / m)
        x[1:-1] = _newton(lambda t: legendre(m, t)[1:], x0)
    p, _, _ = legendre(m, x)
    w = 2.0 / (n * m * p * p)
    return 0.5 * (x + 1.0), 0.5 * w
