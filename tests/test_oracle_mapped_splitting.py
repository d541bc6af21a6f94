"""Pins of the oracle's splitting step on trilinear cells (CPU, no GPU).

Sec. 3.2 / 5.1, Alg. 1 on the general hexahedra of Sec. 5 (the jittered
backward-facing-step channel). Each pin is fixed by the exactness of the forms
for fields the trilinear space represents exactly, or by the affine oracle's
own pins:

* without jitter the trilinear step equals the affine step on the channel
  (inflow ramp, outflow, walls, periodic direction, Carreau viscosity, BDF1 then
  BDF2) - every per-point geometry term reduces to its affine constant;
* a uniform flow with matching wall data is preserved exactly on a jittered box
  (the convective, pressure, projection and viscous forms of a constant field
  vanish or cancel for any cell shape) and the pressure stays zero;
* a fluid at rest under a constant body force keeps u = 0 and gets the linear
  hydrostatic pressure on a jittered box (pure Neumann pressure, mean-free) and
  on the jittered channel with the outflow at p = 0: a linear function of x is
  in the mapped pressure space of trilinear cells.
A dropped det J, a transposed J^-1, a normal taken from the reference face or a
wrong surface weight breaks the preservation or the reduction.
"""
import numpy as np

from oracle import splitting as osp
from oracle.mapped import MappedMesh, MappedSIPG, jittered_vertices
from oracle.mesh import BoxMesh
from paper_2506_14424_gb300 import inputs

VEL_BC = ('D', 'N', 'D', 'D', 'D', 'D', 'D')   # inflow, outflow, walls, (z periodic), step


def _channel():
    return inputs.bfs_channel(2, inlet_length=1.0, outlet_length=3.0, depth=1.0)


def test_unjittered_trilinear_step_equals_affine_step():
    c = _channel()
    flat = inputs.bfs_vertices(c, amp=0.0)
    mm = MappedMesh(*c["dims"], flat, bc=VEL_BC, active=c["active"], periodic=c["periodic"])
    bm = BoxMesh(*c["dims"], extent=c["extent"], lo=c["lo"], active=c["active"], periodic=c["periodic"], bc=VEL_BC)
    k = 2
    rh = inputs.carreau_blood_like()
    inflow = [lambda x: np.stack([1.0 - ((x[:, 1] - 1.5) / 0.5) ** 2, 0 * x[:, 0], 0 * x[:, 0]], axis=1)]
    g = inflow + [np.zeros(3)] * 6
    ramp = lambda t: np.sin(np.pi * t / 2.0) ** 2  # noqa: E731
    runs = []
    for mesh in (bm, mm):
        sp = osp.Splitting(mesh, k, rh, g_faces=g, ramp=ramp, t0=0.3)
        u0 = sp.Su.interpolate(lambda x: np.stack([0.2 + 0.1 * x[:, 1], 0.05 * x[:, 0], 0 * x[:, 0]], axis=1))
        sp.set_initial(u0)
        runs.append([sp.step(0.02) for _ in range(2)])
    for ra, rm in zip(*runs):
        for key in ('uhat', 'p', 'uhathat', 'u'):
            scale = max(np.abs(ra[key]).max(), 1e-300)
            assert np.abs(ra[key] - rm[key]).max() <= 1e-11 * scale, key


def test_uniform_flow_preserved_on_jittered_cells():
    V = jittered_vertices(2, 2, 2, amp=0.08, seed=7)
    mesh = MappedMesh(2, 2, 2, V)
    U = np.array([0.4, -0.3, 0.2])
    sp = osp.Splitting(mesh, 2, {'law': 'constant', 'nu': 0.05}, g_faces=[U] * 6)
    u0 = sp.Su.interpolate(lambda x: np.broadcast_to(U, x.shape).copy())
    sp.set_initial(u0)
    for _ in range(2):
        out = sp.step(0.05)
        assert np.abs(out['u'] - u0).max() <= 1e-12
        assert np.abs(out['p']).max() <= 1e-11


def test_hydrostatic_state_on_jittered_box():
    V = jittered_vertices(2, 2, 2, amp=0.08, seed=8)
    mesh = MappedMesh(2, 2, 2, V)
    k = 3
    rh = inputs.carreau_blood_like()
    Su = MappedSIPG(mesh, k, 3)
    body = Su.interpolate(lambda x: np.stack([0 * x[:, 0], 0 * x[:, 0], np.ones(len(x))], axis=1))
    sp = osp.Splitting(mesh, k, rh, body=body)
    sp.set_initial(np.zeros(Su.n_dofs))
    pz = MappedSIPG(mesh, k - 1, 1).interpolate(lambda x: x[:, 2])
    pz = pz - pz.mean()
    for _ in range(2):
        out = sp.step(0.02)
        assert np.abs(out['u']).max() <= 1e-12
        assert np.abs(out['p'] - pz).max() <= 1e-11


def test_hydrostatic_outflow_on_jittered_channel():
    c = _channel()
    V = inputs.bfs_vertices(c)
    mesh = MappedMesh(*c["dims"], V, bc=VEL_BC, active=c["active"], periodic=c["periodic"])
    k = 2
    Su = MappedSIPG(mesh, k, 3)
    cb = 0.8
    body = Su.interpolate(lambda x: np.stack([cb + 0 * x[:, 0], 0 * x[:, 0], 0 * x[:, 0]], axis=1))
    sp = osp.Splitting(mesh, k, {'law': 'constant', 'nu': 0.1}, body=body)
    sp.set_initial(np.zeros(Su.n_dofs))
    x_out = c["lo"][0] + c["extent"][0]
    p_exact = MappedSIPG(sp.pmesh, k - 1, 1).interpolate(lambda x: cb * (x[:, 0] - x_out))
    for _ in range(2):
        r = sp.step(0.05)
        assert np.abs(r['u']).max() <= 1e-12
        assert np.abs(r['p'] - p_exact).max() <= 1e-12 * np.abs(p_exact).max()
