"""GPU parity on grids with removed cells and periodic directions (the
backward-facing-step channel: inflow at -x, outflow at +x, walls at +-y and
around the removed block, z periodic) against the oracle.

* node positions (the grid's origin), the viscosity at the points (position
  law and Carreau-Yasuda of a velocity), the viscous operator in FP64,
  float-float and FP32 and the Poisson operator (pressure Dirichlet at the
  outflow) on the channel, degrees 2..4, several CTAs with a ragged tail;
* the multigrid hierarchy: level sizes follow the masked coarsening, the
  transfers and the inverse diagonals equal the oracle's on every level;
* MG-CG solves of the viscous and the (non-singular) pressure problem reach the
  oracle's discrete solution;
* a box periodic in two directions (no removed cell) with the constants in
  the Poisson kernel;
* the splitting step on the channel: boundary faces and their Gauss points;
  BDF1/BDF2 steps with the ramped parabolic inflow (time-dependent wall data
  at the boundary points), the outflow and the Carreau-Yasuda law, with and
  without the penalty step, equal the oracle's; a hydrostatic state with the
  outflow at p = 0 at 448 cells;
* the jittered channel (trilinear cells, 5 % jitter inside the fluid): viscous
  and Poisson applies, the diagonal and the FP64 multigrid solve.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import multigrid as omg  # noqa: E402
from oracle import splitting as osp  # noqa: E402
from oracle.mesh import BoxMesh  # noqa: E402
from oracle.sipg import SIPG  # noqa: E402
from paper_2506_14424_gb300 import Context, inputs  # noqa: E402

pytestmark = pytest.mark.gpu
TOL64 = 1e-12
TOL32 = 2e-5
VEL, PRE = "DNDDDD", "NDNNNN"


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _dev(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def _channel(m):
    return inputs.bfs_channel(m, inlet_length=1.0, outlet_length=3.0, depth=1.0)


def _ctx(c, k, **kw):
    return Context(*c["dims"], k, extent=c["extent"], origin=c["lo"], active=c["active"], periodic=c["periodic"],
                   bc_velocity=VEL, bc_pressure=PRE, bc_removed="DN", **kw)


def _mesh(c, op):
    bc = tuple(VEL) + ('D',) if op == "viscous" else tuple(PRE) + ('N',)
    return BoxMesh(*c["dims"], extent=c["extent"], lo=c["lo"], active=c["active"], periodic=c["periodic"], bc=bc)


def _levels(ctx, op, mesh):
    out = []
    for level in range(ctx.num_levels(op)):
        dims, k, _ = ctx.level_info(op, level)
        if out and tuple(dims) != out[-1][0].n_cells_dir:
            m = out[-1][0].coarsen()
            assert m.n_cells_dir == tuple(dims)
        else:
            m = out[-1][0] if out else mesh
        out.append((m, k))
    return out


def _velocity(S):
    modes = inputs.fourier_modes(1)
    return S.interpolate(lambda p: inputs.fourier_field(p, modes))


@pytest.mark.parametrize("k", [2, 3, 4])
def test_channel_viscous_apply(k):
    c = _channel(2)
    mesh = _mesh(c, "viscous")
    S = SIPG(mesh, k, 3)
    ctx = _ctx(c, k)
    assert ctx.n_dofs("viscous") == S.n_dofs
    pts = ctx.node_points("viscous", 0)
    assert np.abs(pts - np.stack([S.node_points(e) for e in range(mesh.n_cells)])).max() <= 1e-14
    x = inputs.uniform_vector(S.n_dofs, seed=11)
    for rheo, u in (({'law': 'analytic'}, None), (inputs.carreau_blood_like(), _velocity(S))):
        ctx.set_viscosity(rheo, None if u is None else _dev(u))
        nc, nf = ctx.get_viscosity(0)
        rc, rf = S.viscosity_at_points(rheo, u)
        assert _rel(nc.cpu().numpy(), rc) <= 1e-13
        assert _rel(nf.cpu().numpy(), rf) <= 1e-13
        ref = S.apply(x, rc, rf)
        for arith in ("f64", "f64ff"):
            assert _rel(ctx.apply("viscous", _dev(x), arith=arith).cpu().numpy(), ref) <= TOL64, arith
        ref_m = S.apply(x, rc, rf, mass=25.0)
        assert _rel(ctx.apply("viscous", _dev(x), mass=25.0, arith="f64ff").cpu().numpy(), ref_m) <= TOL64
        y32 = ctx.apply("viscous", _dev(x, torch.float32)).double().cpu().numpy()
        assert _rel(y32, ref) <= TOL32
    ctx.close()


@pytest.mark.parametrize("kp", [1, 2, 3])
def test_channel_poisson_apply(kp):
    c = _channel(2)
    P = SIPG(_mesh(c, "poisson"), kp, 1)
    ctx = _ctx(c, kp + 1)
    x = inputs.uniform_vector(P.n_dofs, seed=12)
    ref = P.apply(x)
    for arith in ("f64", "f64ff"):
        assert _rel(ctx.apply("poisson", _dev(x), arith=arith).cpu().numpy(), ref) <= TOL64
    assert _rel(ctx.apply("poisson", _dev(x, torch.float32)).double().cpu().numpy(), ref) <= TOL32
    ctx.close()


@pytest.mark.parametrize("op", ["viscous", "poisson"])
def test_channel_hierarchy_transfers_and_diagonals(op):
    c = _channel(4)   # 16 x 8 x 4 grid, 448 cells; h-levels down to 8 x 4 x 2
    k = 2 if op == "viscous" else 3
    ctx = _ctx(c, k, coarse_max_dofs=500)
    rheo = {'law': 'analytic'}
    ctx.set_viscosity(rheo)
    levels = _levels(ctx, op, _mesh(c, op))
    assert [m.n_cells for m, _ in levels][-1] == _mesh(_channel(2), op).n_cells
    nc = 3 if op == "viscous" else 1
    nus = omg.level_viscosity(levels, rheo) if op == "viscous" else None
    for level, (m, kl) in enumerate(levels):
        S = SIPG(m, kl, nc)
        A = S.assemble(*nus[level]) if op == "viscous" else S.assemble()
        dinv = ctx.inverse_diagonal(op, level).cpu().numpy()
        assert _rel(1.0 / dinv, A.diagonal()) <= TOL64, level
        if level == 0:
            continue
        F, kf = levels[level - 1]
        P = (omg.prolongation_p(m, kf, kl, nc) if F.n_cells == m.n_cells
             else omg.prolongation_h(F, m, kl, nc))
        xc = inputs.uniform_vector(P.shape[1], seed=30 + level)
        xf = inputs.uniform_vector(P.shape[0], seed=40 + level)
        assert _rel(ctx.transfer(op, level - 1, +1, _dev(xc)).cpu().numpy(), P @ xc) <= 1e-14
        assert _rel(ctx.transfer(op, level - 1, -1, _dev(xf)).cpu().numpy(), P.T @ xf) <= 1e-14
    ctx.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_channel_mg_solves(prec):
    c = _channel(2)
    k = 3
    ctx = _ctx(c, k, mg_precision=prec, coarse_max_dofs=2000)
    S = SIPG(_mesh(c, "viscous"), k, 3)
    rheo = inputs.carreau_blood_like()
    u = _velocity(S)
    ctx.set_viscosity(rheo, _dev(u))
    A = S.assemble(*S.viscosity_at_points(rheo, u), mass=40.0)
    u_star = inputs.uniform_vector(S.n_dofs, seed=80)
    b = A @ u_star
    x, st = ctx.solve("viscous", _dev(b), rtol=1e-10, precond="mg", maxit=300, mass=40.0)
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1e-10 * (1 + 1e-6) * np.linalg.norm(b)
    assert st["iterations"] < 60, st
    P = SIPG(_mesh(c, "poisson"), k - 1, 1)
    Ap = P.assemble()
    p_star = inputs.uniform_vector(P.n_dofs, seed=81)
    bp = Ap @ p_star
    xp, st = ctx.solve("poisson", _dev(bp), rtol=1e-10, precond="mg", maxit=300)
    assert _rel(xp.cpu().numpy(), p_star) <= 1e-7
    assert st["iterations"] < 60, st
    ctx.close()


def test_periodic_box():
    """x and z periodic, walls at +-y (velocity Dirichlet, pressure Neumann)."""
    dims, k = (4, 2, 3), 3
    ctx = Context(*dims, k, periodic=(True, False, True))
    mesh = BoxMesh(*dims, periodic=(True, False, True), bc=('N',) * 6)
    P = SIPG(mesh, k - 1, 1)
    x = inputs.uniform_vector(P.n_dofs, seed=5)
    assert _rel(ctx.apply("poisson", _dev(x), arith="f64ff").cpu().numpy(), P.apply(x)) <= TOL64
    ones = torch.ones(P.n_dofs, dtype=torch.float64, device="cuda")
    assert ctx.apply("poisson", ones).abs().max().item() <= 1e-12
    S = SIPG(mesh.with_bc(('D',) * 6), k, 3)
    ctx.set_viscosity({'law': 'analytic'})
    xv = inputs.uniform_vector(S.n_dofs, seed=6)
    ref = S.apply(xv, *S.viscosity_at_points({'law': 'analytic'}))
    assert _rel(ctx.apply("viscous", _dev(xv)).cpu().numpy(), ref) <= TOL64
    ctx.close()


CARREAU = {'law': 'carreau', 'eta0': 1.0, 'eta_inf': 1e-3, 'kappa': 1.0, 'lam': 1.0, 'a': 2.0, 'b': 0.5}


def _inflow(x):
    """Parabolic inflow on the inlet y in [1, 2] (maximum 1 on its centre line)."""
    return np.stack([1 - ((x[:, 1] - 1.5) / 0.5) ** 2, 0 * x[:, 0], 0 * x[:, 0]], axis=1)


def _ramp(t, t_ramp=0.1):
    return np.sin(np.pi * t / (2 * t_ramp)) ** 2 if t < t_ramp else 1.0


def _wall_points(ctx, t):
    ids = ctx.boundary_faces()[:, 2]
    pts = ctx.boundary_points().cpu().numpy()
    g = np.zeros_like(pts)
    inlet = ids == 0
    g[inlet] = _ramp(t) * _inflow(pts[inlet].reshape(-1, 3)).reshape(pts[inlet].shape)
    return _dev(g)


def test_channel_boundary_faces():
    c = _channel(2)
    k = 2
    ctx = _ctx(c, k)
    mesh = _mesh(c, "viscous")
    ref = mesh.boundary_faces()
    got = ctx.boundary_faces()
    assert [(int(e), int(f)) for e, f, _ in got] == ref
    assert [int(b) for b in got[:, 2]] == [mesh.boundary_id(e, f) for e, f in ref]
    S = SIPG(mesh, k, 3)
    pts = ctx.boundary_points().cpu().numpy()
    for i, (e, f) in enumerate(ref):
        assert np.abs(pts[i] - S.face_points(e, f)).max() <= 1e-14
    ctx.close()


@pytest.mark.parametrize("penalty", [False, True])
def test_channel_steps_match_oracle(penalty):
    """Ramped parabolic inflow, outflow, no-slip walls and step, z periodic, Carreau-Yasuda:
    BDF1 then BDF2 steps equal the oracle's exactly-solved steps."""
    c = _channel(2)
    k = 2
    mesh = _mesh(c, "viscous")
    ref = osp.Splitting(mesh, k, CARREAU, g_faces=[_inflow] + [np.zeros(3)] * 6, ramp=_ramp)
    ref.set_initial(np.zeros(ref.Su.n_dofs))
    ctx = _ctx(c, k)
    ctx.step_init(torch.zeros(ref.Su.n_dofs, dtype=torch.float64, device="cuda"))
    dt, t = 0.02, 0.0
    for n in range(3):
        r = ref.step(dt, penalty=penalty)
        st = ctx.step(CARREAU, dt, wall_points=_wall_points(ctx, t + dt), wall_points_prev=_wall_points(ctx, t),
                      ppe_rtol=1e-13, visc_rtol=1e-13, maxit=3000, penalty=penalty, penalty_rtol=1e-13)
        t += dt
        assert st["order"] == r["order"]
        assert _rel(ctx.step_field("uhat").cpu().numpy(), r["uhat"]) <= 1e-10
        assert _rel(ctx.step_field("p").cpu().numpy(), r["p"]) <= 1e-8
        assert _rel(ctx.step_field("u").cpu().numpy(), r["u"]) <= 1e-8
    ctx.close()


def test_channel_hydrostatic_outflow_at_448_cells():
    """u0 = 0 under b = c e_x with the outflow at p = 0: u stays 0, p = c (x - x_out)
    (the property the oracle's pin establishes), 16 x 8 x 4 grid, k = 3."""
    c = _channel(4)
    k = 3
    ctx = _ctx(c, k)
    n = ctx.n_dofs("viscous")
    cb = 0.8
    body = torch.zeros(n, dtype=torch.float64, device="cuda").view(-1, 3, (k + 1) ** 3)
    body[:, 0] = cb
    ctx.step_init(torch.zeros(n, dtype=torch.float64, device="cuda"))
    pp = ctx.node_points("poisson", 0).reshape(-1, 3)
    x_out = c["lo"][0] + c["extent"][0]
    p_exact = cb * (pp[:, 0] - x_out)
    for _ in range(2):
        ctx.step({'law': 'constant', 'nu': 0.1}, 0.05, body=body.reshape(-1), ppe_rtol=1e-13, visc_rtol=1e-13,
                 maxit=3000)
        assert ctx.step_field("u").abs().max().item() <= 1e-10
        assert _rel(ctx.step_field("p").cpu().numpy(), p_exact) <= 1e-10
    ctx.close()


def _mapped_ctx(c, V, k, **kw):
    return Context(*c["dims"], k, extent=c["extent"], origin=c["lo"], active=c["active"], periodic=c["periodic"],
                   bc_velocity=VEL, bc_pressure=PRE, bc_removed="DN", vertices=V, **kw)


@pytest.mark.parametrize("k", [2, 3])
def test_jittered_channel_applies_and_diagonal(k):
    """The channel with 5 % vertex jitter inside the fluid (trilinear cells): viscous
    (Carreau-Yasuda) and Poisson applies and the viscous diagonal equal the oracle's."""
    from oracle.mapped import MappedMesh, MappedSIPG
    c = _channel(2)
    V = inputs.bfs_vertices(c)
    vm = MappedMesh(*c["dims"], V, bc=tuple(VEL) + ('D',), active=c["active"], periodic=c["periodic"])
    S = MappedSIPG(vm, k, 3)
    u = S.interpolate(lambda p: inputs.fourier_field(p, inputs.fourier_modes(1)))
    nc, nf = S.viscosity_at_points(CARREAU, u)
    ctx = _mapped_ctx(c, V, k)
    ctx.set_viscosity(CARREAU, _dev(u))
    x = inputs.uniform_vector(S.n_dofs, seed=21)
    A = S.assemble(nc, nf)
    assert _rel(ctx.apply("viscous", _dev(x)).cpu().numpy(), A @ x) <= TOL64
    assert _rel(ctx.inverse_diagonal("viscous", 0).cpu().numpy(), 1.0 / A.diagonal()) <= TOL64
    pm = MappedMesh(*c["dims"], V, bc=tuple(PRE) + ('N',), active=c["active"], periodic=c["periodic"])
    P = MappedSIPG(pm, k - 1, 1)
    xp = inputs.uniform_vector(P.n_dofs, seed=22)
    assert _rel(ctx.apply("poisson", _dev(xp)).cpu().numpy(), P.assemble() @ xp) <= TOL64
    ctx.close()


def test_jittered_channel_multigrid_solve():
    """FP64 hp-multigrid on the jittered channel (p-levels on the fine vertices, an h-level
    from every other vertex) preconditions CG to the oracle's sparse-LU solution."""
    import scipy.sparse.linalg as spla

    from oracle.mapped import MappedMesh, MappedSIPG
    c = inputs.bfs_channel(2, inlet_length=1.0, outlet_length=3.0, depth=2.0)   # 8 x 4 x 4 grid, 112 cells
    V = inputs.bfs_vertices(c)
    k, m = 2, 5.0
    vm = MappedMesh(*c["dims"], V, bc=tuple(VEL) + ('D',), active=c["active"], periodic=c["periodic"])
    S = MappedSIPG(vm, k, 3)
    u = S.interpolate(lambda p: inputs.fourier_field(p, inputs.fourier_modes(1)))
    nc, nf = S.viscosity_at_points(CARREAU, u)
    b = inputs.uniform_vector(S.n_dofs, 23)
    ref = spla.spsolve(S.assemble(nc, nf, mass=m).tocsc(), b)
    ctx = _mapped_ctx(c, V, k, coarse_max_dofs=2000)
    assert ctx.num_levels("viscous") >= 3
    ctx.set_viscosity(CARREAU, _dev(u))
    xs, st = ctx.solve("viscous", _dev(b), rtol=1e-12, maxit=300, precond="mg", mass=m)
    assert _rel(xs.cpu().numpy(), ref) <= 1e-9
    assert st["iterations"] <= 60, st
    ctx.close()


def _jittered(c):
    from oracle.mapped import MappedMesh
    V = inputs.bfs_vertices(c)
    return V, MappedMesh(*c["dims"], V, bc=tuple(VEL) + ('D',), active=c["active"], periodic=c["periodic"])


def test_jittered_channel_forms_match_oracle():
    """Trilinear cells: the cell mass matrix and its inverse (w det J per point), the
    convective vector with the inflow data, the projection right-hand side and the CFL
    time step equal the oracle's on the jittered channel."""
    from oracle import mass as omass
    from oracle.mapped import MappedSIPG
    c = _channel(2)
    V, mesh = _jittered(c)
    k = 3
    S = MappedSIPG(mesh, k, 3)
    ctx = _mapped_ctx(c, V, k)
    u = S.interpolate(lambda p: inputs.fourier_field(p, inputs.fourier_modes(2)))
    du = _dev(u)
    assert _rel(ctx.mass("viscous", du, coeff=2.5).cpu().numpy(), omass.apply_mass(S, u, 2.5)) <= TOL64
    assert _rel(ctx.mass("viscous", du, coeff=2.5, inverse=True).cpu().numpy(),
                omass.apply_inverse_mass(S, u, 2.5)) <= 1e-11
    assert _rel(ctx.convective(du).cpu().numpy(), osp.convective_vector(S, u, [np.zeros(3)] * 7)) <= TOL64
    Sp = MappedSIPG(mesh, k - 1, 1, n_quad=k + 1)
    p = inputs.uniform_vector(Sp.n_dofs, seed=5)
    assert _rel(ctx.projection_rhs(_dev(p)).cpu().numpy(), osp.projection_rhs(S, Sp, p)) <= TOL64
    assert abs(ctx.cfl_dt(du, 0.3) - osp.cfl_dt(S, u, 0.3)) <= 1e-12 * osp.cfl_dt(S, u, 0.3)
    ctx.close()


def test_jittered_channel_steps_match_oracle():
    """The splitting step on trilinear cells (5 % jitter inside the fluid): ramped parabolic
    inflow, outflow, no-slip walls and step, z periodic, Carreau-Yasuda; BDF1 then BDF2 steps
    equal the oracle's exactly-solved steps."""
    c = _channel(2)
    V, mesh = _jittered(c)
    k = 2
    ref = osp.Splitting(mesh, k, CARREAU, g_faces=[_inflow] + [np.zeros(3)] * 6, ramp=_ramp)
    ref.set_initial(np.zeros(ref.Su.n_dofs))
    ctx = _mapped_ctx(c, V, k)
    ctx.step_init(torch.zeros(ref.Su.n_dofs, dtype=torch.float64, device="cuda"))
    dt, t = 0.02, 0.0
    for n in range(3):
        r = ref.step(dt)
        st = ctx.step(CARREAU, dt, wall_points=_wall_points(ctx, t + dt), wall_points_prev=_wall_points(ctx, t),
                      ppe_rtol=1e-13, visc_rtol=1e-13, maxit=3000)
        t += dt
        assert st["order"] == r["order"]
        assert _rel(ctx.step_field("uhat").cpu().numpy(), r["uhat"]) <= 1e-10
        assert _rel(ctx.step_field("p").cpu().numpy(), r["p"]) <= 1e-8
        assert _rel(ctx.step_field("u").cpu().numpy(), r["u"]) <= 1e-8
    ctx.close()
