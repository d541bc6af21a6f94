"""Pins of the oracle's viscosity laws (CPU, no GPU).

Eq. (viscosity_general) of the paper: eta(gdot) = eta_inf + (eta_0 - eta_inf)
(kappa + (lambda gdot)^a)^((b - 1)/a), with the shear rate gdot = sqrt(2 eps:eps)
of the problem formulation (Sec. 2), eps = sym grad u. Each value below is
fixed by the formula's limits, by a closed-form interior point or by the
kinematics of a textbook flow, not by re-running the oracle's expression:
a dropped exponent denominator, sqrt(eps:eps/2) instead of sqrt(2 eps:eps),
a missing symmetrisation or a transposed gradient each fail one of them.
"""
import numpy as np
import pytest

from oracle import viscosity
from oracle.mesh import BoxMesh
from oracle.sipg import SIPG

GN = viscosity.generalized_newtonian


def test_law_at_zero_shear_is_eta0():
    assert GN(0.0, 1.0, 1e-3, 1.0, 1.0, 2.0, 0.5) == pytest.approx(1.0, rel=1e-15)
    assert GN(0.0, 3.5, 0.2, 1.0, 7.0, 1.3, 0.25) == pytest.approx(3.5, rel=1e-15)


def test_law_at_infinite_shear_is_eta_inf():
    # b < 1: the bracket grows without bound and its negative power vanishes like
    # (lambda gdot)^(b - 1), so the excess over eta_inf decays with that power
    for gdot in (1e8, 1e12):
        eta = GN(gdot, 1.0, 1e-3, 1.0, 1.0, 2.0, 0.5)
        assert eta > 1e-3
        assert (eta - 1e-3) / (1.0 - 1e-3) * gdot ** 0.5 == pytest.approx(1.0, rel=1e-9)
    assert GN(1e30, 1.0, 1e-3, 1.0, 1.0, 2.0, 0.5) == pytest.approx(1e-3, rel=1e-12)


def test_equal_limits_give_a_constant():
    g = np.logspace(-6, 6, 25)
    assert np.all(GN(g, 0.7, 0.7, 1.0, 2.0, 2.0, 0.3) == 0.7)


def test_interior_closed_form_value():
    # kappa = 1, a = 2, b = 1/2, lambda gdot = 1: (1 + 1)^(-1/4)
    eta0, einf = 1.0, 1e-3
    expect = einf + (eta0 - einf) * 2.0 ** -0.25
    assert GN(0.5, eta0, einf, 1.0, 2.0, 2.0, 0.5) == pytest.approx(expect, rel=1e-15)
    # classic Carreau (b = 0, a = 2): (1 + 3)^(-1/2) = 1/2 at lambda gdot = sqrt(3)
    assert GN(np.sqrt(3.0), 2.0, 0.0, 1.0, 1.0, 2.0, 0.0) == pytest.approx(1.0, rel=1e-15)


def test_kappa_zero_is_the_power_law_for_any_a():
    # (lambda gdot)^(a (b-1)/a) = (lambda gdot)^(b-1): the exponent's denominator a cancels
    for a in (0.5, 1.0, 2.0, 3.0):
        assert GN(4.0, 1.0, 0.0, 0.0, 1.0, a, 0.5) == pytest.approx(0.5, rel=1e-14)


def test_shear_rate_of_simple_shear_is_the_shear_gradient():
    for gam in (0.3, -2.5):
        G = np.zeros((3, 3))
        G[0, 1] = gam  # u = (gam y, 0, 0)
        assert viscosity.shear_rate(G) == pytest.approx(abs(gam), rel=1e-15)
        assert viscosity.shear_rate(G.T) == pytest.approx(abs(gam), rel=1e-15)


def test_shear_rate_of_planar_extension():
    e = 0.8
    G = np.diag([e, -e, 0.0])  # u = (e x, -e y, 0)
    assert viscosity.shear_rate(G) == pytest.approx(2.0 * e, rel=1e-15)


def test_rigid_rotation_has_no_shear():
    w = np.array([0.3, -1.2, 2.0])
    G = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])  # u = w x x
    assert viscosity.shear_rate(G) == pytest.approx(0.0, abs=1e-15)


def test_shear_rate_is_frame_invariant():
    rng = np.random.default_rng(11)
    G = rng.standard_normal((3, 3))
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    assert viscosity.shear_rate(Q @ G @ Q.T) == pytest.approx(viscosity.shear_rate(G), rel=1e-13)


def test_analytic_field_values():
    f = viscosity.analytic_field
    assert f(np.array([0.5, 0.5, 0.5])) == pytest.approx(10.0, rel=1e-15)
    assert f(np.array([0.25, 0.5, 0.5])) == pytest.approx(5.5, rel=1e-14)  # sin^2(pi/4) = 1/2
    for p in ([0.0, 0.3, 0.7], [0.4, 1.0, 0.2], [0.6, 0.1, 0.0]):
        assert f(np.array(p)) == pytest.approx(1.0, abs=1e-14)


def test_sinker_field_inside_outside_and_on_the_surface():
    c = np.array([[0.5, 0.5, 0.5], [0.125, 0.125, 0.125]])
    pts = np.array([[0.75, 0.5, 0.5],          # exactly on the first sphere (r = 1/4): inside
                    [0.5, 0.5, 0.5],           # centre
                    [0.7500001, 0.5, 0.5],     # just outside
                    [0.125, 0.125, 0.375],     # exactly on the second sphere
                    [0.9, 0.9, 0.9]])
    nu = viscosity.sinker_field(pts, c, 0.25, 1e4, 1.0)
    assert list(nu) == [1e4, 1e4, 1.0, 1e4, 1.0]


@pytest.mark.parametrize("k", [2, 3])
def test_carreau_of_interpolated_simple_shear_at_every_point(k):
    """u = (gam y, 0, 0) is in Q_k, so its interpolant's gradient is exact at every
    cell and face point of every cell, and nu must equal eta(|gam|) there (both
    sides of each face): pins the gradient, the shear rate and the law together."""
    gam = 1.7
    rh = {'law': 'carreau', 'eta0': 1.0, 'eta_inf': 1e-3, 'kappa': 1.0, 'lam': 1.0, 'a': 2.0, 'b': 0.5}
    S = SIPG(BoxMesh(3, 2, 2, extent=(1.5, 0.5, 0.8)), k, 3)
    u = S.interpolate(lambda p: np.stack([gam * p[:, 1], 0 * p[:, 0], 0 * p[:, 0]], axis=1))
    nc, nf = S.viscosity_at_points(rh, u)
    expect = 1e-3 + (1.0 - 1e-3) * (1.0 + gam * gam) ** -0.25
    assert np.max(np.abs(nc - expect)) <= 1e-13
    assert np.max(np.abs(nf - expect)) <= 1e-13


def test_carreau_of_interpolated_extension_flow():
    """u = (e x, -e y, 0): gdot = 2|e| everywhere, eta from the closed form."""
    e = 0.4
    rh = {'law': 'carreau', 'eta0': 2.0, 'eta_inf': 0.1, 'kappa': 1.0, 'lam': 0.5, 'a': 2.0, 'b': 0.5}
    S = SIPG(BoxMesh(2, 2, 3), 2, 3)
    u = S.interpolate(lambda p: np.stack([e * p[:, 0], -e * p[:, 1], 0 * p[:, 0]], axis=1))
    nc, nf = S.viscosity_at_points(rh, u)
    expect = 0.1 + 1.9 * (1.0 + (0.5 * 2 * e) ** 2) ** -0.25
    assert np.max(np.abs(nc - expect)) <= 1e-13 and np.max(np.abs(nf - expect)) <= 1e-13
