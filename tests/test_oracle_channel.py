"""Pins for the oracle on grids with removed cells and periodic directions (the
backward-facing-step channel; Sec. 5 meshes of hexahedra, Sec. 7 geometry).

* topology: cell and boundary-face counts of the channel in closed form; every
  interior face is seen from both sides; the periodic direction has no
  boundary faces;
* a grid whose active cells form a box equals the plain box: the SIPG
  operators agree entry by entry after renumbering (faces against removed cells
  take the type of the box side they replace) - this pins the removed-cell
  faces and the numbering against the box oracle's own pins;
* periodic direction: the operators commute with the shift by one cell layer,
  and with every side periodic or Neumann the constants (Poisson) and rigid
  translations (viscous) stay in the kernel;
* channel operators: symmetric; positive definite with the channel's walls
  (velocity Dirichlet on inflow and walls, Neumann outflow; pressure Dirichlet
  outflow); Galerkin consistency A u_I = D(g = u) for a linear velocity with zero
  traction on the outflow;
* multigrid on the channel: the h-prolongation reproduces a coarse continuous
  polynomial exactly, and the masked coarsening keeps the step.
"""
import numpy as np
import pytest

from oracle import multigrid as omg
from oracle import splitting as osp
from oracle.mesh import BoxMesh
from oracle.sipg import SIPG
from paper_2506_14424_gb300 import inputs

VEL_BC = ('D', 'N', 'D', 'D', 'D', 'D', 'D')   # inflow, outflow, walls, (z periodic), step
PRE_BC = ('N', 'D', 'N', 'N', 'N', 'N', 'N')


def small_channel(m=2, bc=VEL_BC):
    c = inputs.bfs_channel(m, inlet_length=1.0, outlet_length=3.0, depth=1.0)
    return BoxMesh(*c["dims"], extent=c["extent"], lo=c["lo"], active=c["active"], periodic=c["periodic"], bc=bc)


def test_channel_topology_counts():
    m = 2
    mesh = small_channel(m)
    nx, ny, nz = mesh.n_cells_dir
    assert (nx, ny, nz) == (8, 4, 2)
    removed = (1 * m) * (1 * m) * nz
    assert mesh.n_cells == nx * ny * nz - removed
    faces = mesh.boundary_faces()
    ids = [mesh.boundary_id(e, f) for e, f in faces]
    # inflow: the inlet's cross-section; outflow: the full height; walls
    assert ids.count(0) == (2 - 1) * m * nz
    assert ids.count(1) == 2 * m * nz
    assert ids.count(2) == 3 * m * nz          # bottom wall behind the step
    assert ids.count(3) == 4 * m * nz          # top wall over the whole length
    assert ids.count(6) == (1 * m + 1 * m) * nz  # step face x = 0 and inlet floor y = 1
    assert ids.count(4) == ids.count(5) == 0   # z periodic
    for e in range(mesh.n_cells):
        for f in range(6):
            nb = mesh.neighbor(e, f)
            if nb is not None:
                assert mesh.neighbor(nb, f ^ 1) == e


@pytest.mark.parametrize("ncomp,k", [(3, 2), (1, 2)])
def test_masked_box_equals_plain_box(ncomp, k):
    # active cells x >= 0.5 of a 4x2x2 grid: the box [0.5, 1] x [0, 1] x [0, 1]
    bc = ('N', 'D', 'D', 'N', 'D', 'D')
    act = np.zeros((2, 2, 4), dtype=bool)
    act[:, :, 2:] = True
    masked = BoxMesh(4, 2, 2, bc=bc + (bc[0],), active=act)
    plain = BoxMesh(2, 2, 2, extent=(0.5, 1.0, 1.0), bc=bc)
    assert masked.n_cells == plain.n_cells
    rh = {'law': 'constant', 'nu': 0.7}
    Sm, Sp = SIPG(masked, k, ncomp), SIPG(plain, k, ncomp)
    Am = Sm.assemble(*Sm.viscosity_at_points(rh)) if ncomp == 3 else Sm.assemble()
    Ap = Sp.assemble(*Sp.viscosity_at_points(rh)) if ncomp == 3 else Sp.assemble()
    assert np.abs((Am - Ap).toarray()).max() <= 1e-13 * np.abs(Ap.toarray()).max()
    # positions: the masked mesh's cell e sits where the plain mesh's cell e does, shifted
    assert np.allclose(Sm.node_points(0) - np.array([0.5, 0, 0]), Sp.node_points(0), atol=1e-15)


@pytest.mark.parametrize("ncomp", [1, 3])
def test_periodic_shift_invariance_and_kernel(ncomp):
    mesh = BoxMesh(2, 2, 4, bc=('N',) * 6, periodic=(False, False, True))
    S = SIPG(mesh, 2, ncomp)
    A = (S.assemble(*S.viscosity_at_points({'law': 'constant', 'nu': 1.0})) if ncomp == 3 else S.assemble()).toarray()
    m = ncomp * 27
    perm = np.zeros(mesh.n_cells, dtype=int)
    for e in range(mesh.n_cells):
        i, j, k = mesh.cell_ijk(e)
        perm[e] = mesh.cell_index((i, j, (k + 1) % 4))
    P = np.zeros_like(A)
    for e in range(mesh.n_cells):
        P[perm[e] * m:(perm[e] + 1) * m, e * m:(e + 1) * m] = np.eye(m)
    assert np.abs(P @ A @ P.T - A).max() <= 1e-12 * np.abs(A).max()
    for c in range(ncomp):
        v = S.interpolate(lambda x: np.eye(ncomp)[c][None, :].repeat(len(x), 0) if ncomp == 3 else np.ones(len(x)))
        assert np.abs(A @ v).max() <= 1e-12 * np.abs(A).max()


def test_channel_operators_spd():
    mesh = small_channel(2)
    S = SIPG(mesh, 2, 3)
    A = S.assemble(*S.viscosity_at_points({'law': 'constant', 'nu': 0.3})).toarray()
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0
    Sp = SIPG(mesh.with_bc(PRE_BC), 1, 1)
    Ap = Sp.assemble().toarray()
    assert np.abs(Ap - Ap.T).max() <= 1e-13 * np.abs(Ap).max()
    assert np.linalg.eigvalsh(Ap).min() > 0


def test_channel_dirichlet_consistency():
    """u = (0, 0, c y): linear, periodic in z, zero traction 2 nu eps(u) n on the outflow
    (normal e_x); A u_I equals the Dirichlet data terms of u on inflow, walls and step."""
    mesh = small_channel(2)
    S = SIPG(mesh, 2, 3)
    ufn = lambda x: np.stack([0 * x[:, 0], 0 * x[:, 0], 0.7 * x[:, 1]], axis=1)
    nc, nf = S.viscosity_at_points({'law': 'constant', 'nu': 1.3})
    u = S.interpolate(ufn)
    lhs = S.apply(u, nc, nf)
    D = osp.viscous_dirichlet_rhs(S, nf, [ufn] * 7)
    assert np.abs(lhs - D).max() <= 1e-12 * np.abs(D).max()


def test_channel_multigrid_transfer():
    mesh = small_channel(4)
    coarse = mesh.coarsen()
    assert coarse.n_cells_dir == (8, 4, 2) and coarse.n_cells == small_channel(2).n_cells
    with pytest.raises(ValueError):
        coarse.coarsen()   # the step height is one coarse cell
    k = 2
    P = omg.prolongation_h(mesh, coarse, k, 1)
    poly = lambda x: 1 + x[:, 0] - 2 * x[:, 1] ** 2 + x[:, 0] * x[:, 2]
    uc = SIPG(coarse, k, 1).interpolate(poly)
    uf = SIPG(mesh, k, 1).interpolate(poly)
    assert np.abs(P @ uc - uf).max() <= 1e-13


def test_channel_hydrostatic_with_outflow():
    """u0 = 0 under a uniform body force b = c e_x, no-slip walls and step, zero inflow,
    outflow traction-free with p = 0: BDF1 and BDF2 steps keep u = 0 and give p = c (x - x_out)
    (the PPE's outflow face term (q, uhat.n) with uhat = dt/gamma0 b, the pressure Dirichlet
    condition and the non-singular pressure solve)."""
    mesh = small_channel(2)
    k = 2
    S = SIPG(mesh, k, 3)
    c = 0.8
    body = S.interpolate(lambda x: np.stack([c + 0 * x[:, 0], 0 * x[:, 0], 0 * x[:, 0]], axis=1))
    ref = osp.Splitting(mesh, k, {'law': 'constant', 'nu': 0.1}, body=body)
    ref.set_initial(np.zeros(S.n_dofs))
    Sp = SIPG(mesh.with_bc(PRE_BC), k - 1, 1)
    x_out = mesh.lo[0] + mesh.extent[0]
    p_exact = Sp.interpolate(lambda x: c * (x[:, 0] - x_out))
    for _ in range(2):
        r = ref.step(0.05)
        assert np.abs(r['u']).max() <= 1e-12
        assert np.abs(r['p'] - p_exact).max() <= 1e-12 * np.abs(p_exact).max()


def test_ppe_datum_depends_on_the_newest_wall_data_only():
    """h_p - (gamma0/dt) g_uhat.n with the BDF approximation of d_t g: the older wall data
    cancel (-(gamma0/dt) n.g(t_{n+1}) is the only wall term)."""
    mesh = small_channel(2)
    S = SIPG(mesh, 2, 3)
    rng = np.random.default_rng(3)
    hist = [rng.uniform(-1, 1, S.n_dofs) for _ in range(2)]
    g_new = [rng.uniform(-1, 1, 3) for _ in range(7)]
    g_old = [[rng.uniform(-1, 1, 3) for _ in range(7)] for _ in range(2)]
    e, f = [(e, f) for e, f in mesh.boundary_faces() if mesh.boundary_type(e, f) == 'D'][0]
    rh = {'law': 'constant', 'nu': 0.3}
    a = osp.ppe_boundary_datum(S, e, f, hist, 2, 0.1, None, g_new, rh, g_old)
    b = osp.ppe_boundary_datum(S, e, f, hist, 2, 0.1, None, g_new, rh, None)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    zero = [np.zeros(3)] * 7
    c0 = osp.ppe_boundary_datum(S, e, f, hist, 2, 0.1, None, zero, rh, None)
    _, _, nvec = osp.face_normal(f)
    gn = g_new[mesh.boundary_id(e, f)] @ nvec
    assert np.abs(b - (c0 - 1.5 / 0.1 * gn)).max() <= 1e-12 * np.abs(b).max()


def test_jittered_channel_operators():
    """Trilinear cells on the channel (vertices inside the fluid jittered): symmetric,
    definite with the channel's walls, and equal to the affine channel without jitter."""
    from oracle.mapped import MappedMesh, MappedSIPG
    c = inputs.bfs_channel(2, inlet_length=1.0, outlet_length=3.0, depth=1.0)
    V = inputs.bfs_vertices(c)
    flat = inputs.bfs_vertices(c, amp=0.0)
    assert np.abs(V - flat).max() > 0.01 / 2
    mm = MappedMesh(*c["dims"], V, bc=VEL_BC, active=c["active"], periodic=c["periodic"])
    S = MappedSIPG(mm, 2, 3)
    A = S.assemble(*S.viscosity_at_points({'law': 'constant', 'nu': 0.4})).toarray()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0
    m0 = MappedMesh(*c["dims"], flat, bc=VEL_BC, active=c["active"], periodic=c["periodic"])
    S0 = MappedSIPG(m0, 2, 3)
    A0 = S0.assemble(*S0.viscosity_at_points({'law': 'constant', 'nu': 0.4}))
    Sa = SIPG(small_channel(2), 2, 3)
    Aa = Sa.assemble(*Sa.viscosity_at_points({'law': 'constant', 'nu': 0.4}))
    assert np.abs((A0 - Aa).toarray()).max() <= 1e-12 * np.abs(Aa.toarray()).max()


def test_channel_penalty_step_keeps_a_compatible_field():
    """Eq. (penalty_step) on the channel: u = (0, 0, c y) is continuous, divergence free and
    periodic in z; with its own values as wall data on inflow, walls and step (the
    outflow is Neumann: no term) both penalties vanish and the step returns u."""
    mesh = small_channel(2)
    S = SIPG(mesh, 2, 3)
    ufn = lambda x: np.stack([0 * x[:, 0], 0 * x[:, 0], 0.6 * x[:, 1]], axis=1)
    u = S.interpolate(ufn)
    ut, tdiv, tcon = osp.penalty_step(S, u, 0.2, [ufn] * 7)
    assert np.all(tdiv > 0) and np.all(tcon > 0)
    assert np.abs(ut - u).max() <= 1e-12
