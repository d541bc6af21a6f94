"""GPU parity of the divergence and continuity penalty step (Sec. 3.2,
Eq. penalty_step, the last sub-step of Alg. 1) against the oracle.

* the penalty parameters per cell, the operator K x for random x and random
  parameters, and the wall-data right-hand side, degrees 2, 3, 5 on boxes with
  several cells per direction (interior faces in every direction);
* the post-processed velocity of a divergent, discontinuous field equals the
  oracle's exact sparse solve;
* whole steps (BDF1 then BDF2, lid-driven box, Carreau-Yasuda law) with the
  penalty step switched on equal the oracle's steps;
* at 8^3, k = 3: a uniform flow with matching wall velocity is its own
  post-processed velocity, and the penalty energy of a random field drops;
* an iteration limit that is too small is reported as SIPG_ERR_MAXIT.
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
CASES = [((3, 2, 2), 3, (1.0, 0.8, 0.6)), ((2, 3, 2), 2, (1.0, 1.0, 1.0)), ((2, 2, 1), 5, (0.7, 1.0, 0.5))]


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _field(Su, seed):
    modes = inputs.fourier_modes(seed)
    return Su.interpolate(lambda x: inputs.fourier_field(x, modes)) + 0.2 * inputs.uniform_vector(Su.n_dofs, seed + 1)


@pytest.mark.parametrize("dims,k,ext", CASES)
def test_penalty_forms_match_oracle(dims, k, ext):
    mesh = BoxMesh(*dims, extent=ext)
    Su = SIPG(mesh, k, 3)
    u = _field(Su, 3)
    dt = 0.07
    td_ref, tc_ref = osp.penalty_parameters(Su, u, dt)
    ctx = Context(*dims, k, extent=ext)
    td, tc = ctx.penalty_tau(_dev(u), dt)
    assert _rel(td.cpu().numpy(), td_ref) <= 1e-13
    assert _rel(tc.cpu().numpy(), tc_ref) <= 1e-13
    # the operator for random positive parameters (each term weighs in)
    rng = np.random.default_rng(11)
    tdr, tcr = rng.uniform(0.05, 0.5, mesh.n_cells), rng.uniform(0.05, 0.5, mesh.n_cells)
    x = inputs.uniform_vector(Su.n_dofs, 12)
    ref = osp.penalty_blocks(Su, tdr, tcr) @ x
    y = ctx.penalty_apply(_dev(tdr), _dev(tcr), _dev(x))
    assert _rel(y.cpu().numpy(), ref) <= 1e-13
    wall = np.random.default_rng(5).uniform(-1, 1, size=(6, 3))
    ref = osp.penalty_wall_rhs(Su, tcr, list(wall))
    y = ctx.penalty_wall_rhs(wall, _dev(tcr))
    assert _rel(y.cpu().numpy(), ref) <= 1e-13
    ctx.close()


@pytest.mark.parametrize("dims,k,ext", CASES)
def test_penalty_step_matches_oracle(dims, k, ext):
    mesh = BoxMesh(*dims, extent=ext)
    Su = SIPG(mesh, k, 3)
    u = _field(Su, 7)
    wall = np.random.default_rng(8).uniform(-1, 1, size=(6, 3))
    ref, _, _ = osp.penalty_step(Su, u, 0.3, list(wall))
    ctx = Context(*dims, k, extent=ext)
    ud = _dev(u)
    out, info = ctx.penalty_step(ud, 0.3, wall=wall, rtol=1e-13)
    assert info["rel_residual"] <= 1e-13
    assert info["iterations"] >= 2
    assert _rel(out.cpu().numpy(), ref) <= 1e-11
    # in place
    ctx.penalty_step(ud, 0.3, wall=wall, rtol=1e-13, out=ud)
    assert _rel(ud.cpu().numpy(), ref) <= 1e-11
    ctx.close()


def test_steps_with_penalty_match_oracle():
    dims, k = (3, 2, 2), 2
    mesh = BoxMesh(*dims)
    Su = SIPG(mesh, k, 3)
    modes = inputs.fourier_modes(3)
    u0 = Su.interpolate(lambda x: 0.5 * inputs.fourier_field(x, modes))
    body = Su.interpolate(lambda x: 2.0 * np.stack([np.sin(np.pi * x[:, 2]), 0 * x[:, 0],
                                                    np.cos(np.pi * x[:, 0])], axis=1))
    wall = np.zeros((6, 3))
    wall[5] = (1.0, 0.5, 0.0)
    ref = osp.Splitting(mesh, k, CARREAU, g_faces=list(wall), body=body)
    ref.set_initial(u0)
    ctx = Context(*dims, k)
    ctx.step_init(_dev(u0))
    bd = _dev(body)
    for n in range(3):
        r = ref.step(0.02, penalty=True)
        st = ctx.step(CARREAU, 0.02, wall=wall, body=bd, ppe_rtol=1e-13, visc_rtol=1e-13, maxit=2000,
                      penalty=True, penalty_rtol=1e-13)
        assert st["penalty_iterations"] >= 1
        assert _rel(ctx.step_field("p").cpu().numpy(), r["p"]) <= 1e-8
        assert _rel(ctx.step_field("u").cpu().numpy(), r["u"]) <= 1e-8
    ctx.close()


def test_penalty_properties_at_8cubed():
    N, k = 8, 3
    ctx = Context(N, N, N, k)
    U = np.array([0.4, -0.3, 0.2])
    u0 = torch.tensor(np.broadcast_to(U[None, :, None], (N ** 3, 3, (k + 1) ** 3)).reshape(-1).copy(),
                      device="cuda")
    out, info = ctx.penalty_step(u0, 0.05, wall=np.tile(U, (6, 1)), rtol=1e-13)
    assert (out - u0).abs().max().item() <= 1e-13
    w = u0 + 0.3 * torch.tensor(inputs.uniform_vector(ctx.n_dofs("viscous"), 9), device="cuda")
    td, tc = ctx.penalty_tau(w, 0.5)
    wt, info = ctx.penalty_step(w, 0.5, wall=np.tile(U, (6, 1)), rtol=1e-12)
    assert info["iterations"] >= 2 and info["rel_residual"] <= 1e-12

    def energy(v):  # the penalty part of K: K v - M v, with its wall data
        return float(torch.dot(v, ctx.penalty_apply(td, tc, v) - ctx.mass("viscous", v)))

    # the penalties act on the difference to the wall-compatible uniform state
    assert energy(wt - u0) < energy(w - u0)
    ctx.close()


def test_penalty_status_codes():
    dims, k = (2, 2, 2), 3
    ctx = Context(*dims, k)
    Su = SIPG(BoxMesh(*dims), k, 3)
    ud = _dev(_field(Su, 4))
    with pytest.raises(SipgError):
        ctx.penalty_step(ud, 2.0, rtol=1e-14, maxit=1)
    with pytest.raises(SipgError):
        ctx.penalty_step(ud, 0.0)
    ctx.close()
