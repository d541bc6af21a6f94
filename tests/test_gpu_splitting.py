"""GPU parity of the splitting step (Sec. 3.2 / 5.1, Alg. 1) against the oracle.

* each form on its own: the convective vector with wall velocity, the
  projection right-hand side, the wall-data terms of the viscous step, the CFL
  time step (degrees 2, 3, 5; several cells per direction);
* whole steps (BDF1 then BDF2) on a lid-driven box with a body force and the
  Carreau-Yasuda law: the intermediate velocity, the pressure right-hand side
  (with the consistent Neumann datum), the pressure, the projected velocity
  and the new velocity equal the oracle's exactly-solved step, and the same
  with the implicit (Picard/Aitken) viscosity on no-slip walls;
* at 8^3, k = 3, where the oracle is too slow for a full step: a hydrostatic
  state and a uniform flow are preserved exactly (the properties the oracle's
  own pins establish).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import splitting as osp  # noqa: E402
from oracle.mesh import BoxMesh  # noqa: E402
from oracle.sipg import SIPG  # noqa: E402
from paper_2506_14424_gb300 import Context, SipgError, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

CARREAU = {'law': 'carreau', 'eta0': 1.0, 'eta_inf': 1e-3, 'kappa': 1.0, 'lam': 1.0, 'a': 2.0, 'b': 0.5}


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _walls(seed):
    return np.random.default_rng(seed).uniform(-1, 1, size=(6, 3))


CASES = [((3, 2, 2), 3, (1.0, 0.8, 0.6)), ((2, 3, 2), 2, (1.0, 1.0, 1.0)), ((2, 2, 1), 5, (0.7, 1.0, 0.5))]


@pytest.mark.parametrize("dims,k,ext", CASES)
def test_convective_matches_oracle(dims, k, ext):
    mesh = BoxMesh(*dims, extent=ext)
    Su = SIPG(mesh, k, 3)
    modes = inputs.fourier_modes(3)
    u = Su.interpolate(lambda x: inputs.fourier_field(x, modes)) + 0.1 * inputs.uniform_vector(Su.n_dofs, 4)
    wall = _walls(5)
    ref = osp.convective_vector(Su, u, list(wall))
    ctx = Context(*dims, k, extent=ext)
    y = ctx.convective(_dev(u), wall)
    assert _rel(y.cpu().numpy(), ref) <= 1e-12
    ctx.close()


@pytest.mark.parametrize("dims,k,ext", CASES)
def test_projection_rhs_matches_oracle(dims, k, ext):
    mesh = BoxMesh(*dims, extent=ext)
    Su = SIPG(mesh, k, 3)
    Sp = SIPG(mesh, k - 1, 1, n_quad=k + 1)
    p = inputs.uniform_vector(Sp.n_dofs, 6)
    ref = osp.projection_rhs(Su, Sp, p)
    ctx = Context(*dims, k, extent=ext)
    y = ctx.projection_rhs(_dev(p))
    assert _rel(y.cpu().numpy(), ref) <= 1e-12
    ctx.close()


@pytest.mark.parametrize("dims,k,ext", CASES)
def test_viscous_wall_rhs_and_cfl_match_oracle(dims, k, ext):
    mesh = BoxMesh(*dims, extent=ext)
    Su = SIPG(mesh, k, 3)
    modes = inputs.fourier_modes(3)
    u = Su.interpolate(lambda x: inputs.fourier_field(x, modes))
    nc, nf = Su.viscosity_at_points(CARREAU, u)
    wall = _walls(7)
    ref = osp.viscous_dirichlet_rhs(Su, nf, list(wall))
    ctx = Context(*dims, k, extent=ext)
    ud = _dev(u)
    ctx.set_viscosity(CARREAU, ud)
    y = ctx.viscous_wall_rhs(wall)
    assert _rel(y.cpu().numpy(), ref) <= 1e-12
    assert abs(ctx.cfl_dt(ud, 0.4) - osp.cfl_dt(Su, u, 0.4)) <= 1e-14 * osp.cfl_dt(Su, u, 0.4)
    ctx.close()


def _step_case(dims, k, lid, body_amp, seed=3):
    mesh = BoxMesh(*dims)
    Su = SIPG(mesh, k, 3)
    modes = inputs.fourier_modes(seed)
    u0 = Su.interpolate(lambda x: 0.5 * inputs.fourier_field(x, modes))
    body = Su.interpolate(lambda x: body_amp * np.stack([np.sin(np.pi * x[:, 2]), 0 * x[:, 0],
                                                         np.cos(np.pi * x[:, 0])], axis=1))
    wall = np.zeros((6, 3))
    wall[5] = lid
    return mesh, u0, body, wall


@pytest.mark.parametrize("dims,k", [((3, 2, 2), 2), ((2, 2, 2), 3)])
def test_steps_match_oracle(dims, k):
    mesh, u0, body, wall = _step_case(dims, k, (1.0, 0.5, 0.0), 2.0)
    ref = osp.Splitting(mesh, k, CARREAU, g_faces=list(wall), body=body)
    ref.set_initial(u0)
    ctx = Context(*dims, k)
    ctx.step_init(_dev(u0))
    bd = _dev(body)
    dt = 0.01
    for n in range(3):
        r = ref.step(dt)
        st = ctx.step(CARREAU, dt, wall=wall, body=bd, ppe_rtol=1e-13, visc_rtol=1e-13, maxit=2000)
        assert st["order"] == r["order"] == (1 if n == 0 else 2)
        assert _rel(ctx.step_field("uhat").cpu().numpy(), r["uhat"]) <= 1e-11
        assert _rel(ctx.step_field("ppe_rhs").cpu().numpy(), r["ppe_rhs"]) <= 1e-11
        assert _rel(ctx.step_field("p").cpu().numpy(), r["p"]) <= 1e-8
        assert _rel(ctx.step_field("uhathat").cpu().numpy(), r["uhathat"]) <= 1e-8
        assert _rel(ctx.step_field("u").cpu().numpy(), r["u"]) <= 1e-8
    ctx.close()


def test_implicit_viscosity_step_matches_oracle():
    dims, k = (2, 2, 2), 2
    mesh, u0, body, wall = _step_case(dims, k, (0.0, 0.0, 0.0), 1.0)
    ref = osp.Splitting(mesh, k, CARREAU, body=body, viscosity_mode='implicit')
    ref.set_initial(u0)
    ctx = Context(*dims, k)
    ctx.step_init(_dev(u0))
    bd = _dev(body)
    for n in range(2):
        r = ref.step(0.02, picard={'rtol': 1e-11, 'maxit': 40})
        st = ctx.step(CARREAU, 0.02, body=bd, viscosity_mode="implicit", ppe_rtol=1e-13, maxit=2000,
                      picard={'rtol': 1e-11, 'atol': 0.0, 'maxit': 40, 'lin_rtol': 1e-12, 'lin_maxit': 2000})
        assert st["picard_updates"] >= 2
        assert _rel(ctx.step_field("u").cpu().numpy(), r["u"]) <= 1e-8
    ctx.close()


def test_hydrostatic_and_uniform_states_at_8cubed():
    N, k = 8, 3
    ctx = Context(N, N, N, k)
    n = ctx.n_dofs("viscous")
    body = torch.zeros(n, dtype=torch.float64, device="cuda").view(-1, 3, (k + 1) ** 3)
    body[:, 2] = 1.0
    body = body.reshape(-1)
    ctx.step_init(torch.zeros(n, dtype=torch.float64, device="cuda"))
    Spp = SIPG(BoxMesh(N, N, N), k - 1, 1)
    pz = Spp.interpolate(lambda x: x[:, 2])
    pz -= pz.mean()
    for _ in range(2):
        ctx.step(CARREAU, 0.01, body=body, ppe_rtol=1e-13, visc_rtol=1e-13, maxit=3000)
        assert ctx.step_field("u").abs().max().item() <= 1e-10
        assert _rel(ctx.step_field("p").cpu().numpy(), pz) <= 1e-10
    U = np.array([0.4, -0.3, 0.2])
    u0 = torch.tensor(np.broadcast_to(U[None, :, None], (N ** 3, 3, (k + 1) ** 3)).reshape(-1).copy(),
                      device="cuda")
    ctx.step_init(u0)
    for _ in range(2):
        ctx.step(CARREAU, 0.01, wall=np.tile(U, (6, 1)), ppe_rtol=1e-13, visc_rtol=1e-13, maxit=3000)
        assert (ctx.step_field("u") - u0).abs().max().item() <= 1e-10
    ctx.close()


def test_step_status_codes():
    ctx = Context(2, 2, 2, 2)
    with pytest.raises(SipgError):
        ctx.step(CARREAU, 0.01)  # no state yet
    ctx.step_init(torch.zeros(ctx.n_dofs("viscous"), dtype=torch.float64, device="cuda"))
    with pytest.raises(SipgError):
        ctx.step(CARREAU, -1.0)
    wall = np.zeros((6, 3))
    wall[5, 0] = 1.0
    with pytest.raises(SipgError):
        ctx.step(CARREAU, 0.01, wall=wall, viscosity_mode="implicit")
    with pytest.raises(SipgError):
        ctx.step({'law': 'analytic'}, 0.01)
    ctx.close()
    # a side that is velocity Neumann needs the pressure Dirichlet there (outflow), and a
    # velocity-Dirichlet side the pressure Neumann
    for bv, bp in (("DDDDDN", "NNNNNN"), ("DDDDDD", "NNNNND")):
        c2 = Context(2, 2, 2, 2, bc_velocity=bv, bc_pressure=bp)
        with pytest.raises(SipgError):
            c2.step_init(torch.zeros(c2.n_dofs("viscous"), dtype=torch.float64, device="cuda"))
        c2.close()
    c3 = Context(2, 2, 2, 2, bc_velocity="DDDDDN", bc_pressure="NNNNND")   # outflow at +z
    c3.step_init(torch.zeros(c3.n_dofs("viscous"), dtype=torch.float64, device="cuda"))
    c3.close()
