"""GPU parity of the linearly implicit convective term (alpha_c = 1) and its GMRES solve.

* c_h(., u; w) linear in u, with wall velocity for w and for u, equals the
  oracle's explicit blocks (plus its wall-data vector);
* GMRES on ((m M + A(nu)) + C(w)) x = b, preconditioned by the V-cycle of the
  symmetric part, reaches the oracle's sparse-LU solution;
* BDF1/BDF2 steps with the convective term in the viscous step match the
  oracle's exactly solved steps on a lid-driven box.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")

from oracle import mass as omass  # noqa: E402
from oracle import splitting as osp  # noqa: E402
from oracle.mesh import BoxMesh  # noqa: E402
from oracle.sipg import SIPG  # noqa: E402
from paper_2506_14424_gb300 import Context, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

CARREAU = {'law': 'carreau', 'eta0': 1.0, 'eta_inf': 1e-3, 'kappa': 1.0, 'lam': 1.0, 'a': 2.0, 'b': 0.5}


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("dims,k", [((3, 2, 2), 3), ((2, 3, 2), 2), ((2, 2, 1), 5)])
def test_linearised_convective_matches_oracle(dims, k):
    S = SIPG(BoxMesh(*dims), k, 3)
    rng = np.random.default_rng(8)
    w = S.interpolate(lambda x: inputs.fourier_field(x, inputs.fourier_modes(2)))
    u = rng.uniform(-1, 1, S.n_dofs)
    gw = rng.uniform(-1, 1, (6, 3))
    gu = rng.uniform(-1, 1, (6, 3))
    ref = osp.convective_blocks(S, w, list(gw)) @ u - osp.convective_wall_rhs(S, w, list(gw), list(gu))
    ctx = Context(*dims, k)
    y = ctx.convective_lin(_dev(w), _dev(u), gw, gu)
    assert _rel(y.cpu().numpy(), ref) <= 1e-12
    ctx.close()


def test_gmres_solve_matches_oracle():
    dims, k, m = (3, 2, 2), 3, 40.0
    S = SIPG(BoxMesh(*dims), k, 3)
    w = S.interpolate(lambda x: 3.0 * inputs.fourier_field(x, inputs.fourier_modes(2)))
    nc, nf = S.viscosity_at_points(CARREAU, w)
    K = S.assemble(nc, nf, mass=m) + osp.convective_blocks(S, w, [np.zeros(3)] * 6)
    b = inputs.uniform_vector(S.n_dofs, 9)
    ref = spla.spsolve(K.tocsc(), b)
    ctx = Context(*dims, k, krylov_arith="f64ff")
    wd = _dev(w)
    ctx.set_viscosity(CARREAU, wd)
    x, st = ctx.solve_convective(wd, _dev(b), rtol=1e-12, maxit=400, mass=m, restart=30)
    assert st["status"] == 0 and st["rel_residual"] <= 1.5e-12
    assert _rel(x.cpu().numpy(), ref) <= 1e-9
    # without the convective term it is the symmetric solve
    x2, st2 = ctx.solve_convective(None, _dev(b), rtol=1e-12, maxit=400, mass=m)
    assert st2["status"] == 0 and st2["rel_residual"] <= 1.5e-12
    ref2 = spla.spsolve(S.assemble(nc, nf, mass=m).tocsc(), b)
    assert _rel(x2.cpu().numpy(), ref2) <= 1e-9
    ctx.close()


@pytest.mark.parametrize("dims,k", [((3, 2, 2), 2), ((2, 2, 2), 3)])
def test_linearly_implicit_steps_match_oracle(dims, k):
    mesh = BoxMesh(*dims)
    Su = SIPG(mesh, k, 3)
    u0 = Su.interpolate(lambda x: 0.5 * inputs.fourier_field(x, inputs.fourier_modes(3)))
    body = Su.interpolate(lambda x: np.stack([np.sin(np.pi * x[:, 2]), 0 * x[:, 0], np.cos(np.pi * x[:, 0])],
                                             axis=1))
    wall = np.zeros((6, 3))
    wall[5] = (1.0, 0.5, 0.0)
    ref = osp.Splitting(mesh, k, CARREAU, g_faces=list(wall), body=body, convective='linear_implicit')
    ref.set_initial(u0)
    ctx = Context(*dims, k)
    ctx.step_init(_dev(u0))
    bd = _dev(body)
    for n in range(3):
        r = ref.step(0.02)
        ctx.step(CARREAU, 0.02, wall=wall, body=bd, ppe_rtol=1e-13, visc_rtol=1e-13, maxit=2000,
                 convective_mode="linear_implicit")
        assert _rel(ctx.step_field("uhathat").cpu().numpy(), r["uhathat"]) <= 1e-8
        assert _rel(ctx.step_field("u").cpu().numpy(), r["u"]) <= 1e-8
    ctx.close()
