"""GPU parity of the cell mass operators and the Picard/Aitken viscous step.

* y = coeff M x and y = (coeff M)^-1 x equal the oracle's explicit cell blocks
  (several CTAs with a ragged last one; FP64 and float-float to 1e-13, FP32 to
  single precision), also in place, and on sampled cells at 32^3, k = 3;
* the Picard/Aitken loop takes the oracle's iterates: same number of updates,
  the same residual norms and relaxation factors, the same converged velocity
  (the linear solves run to a tight tolerance so that both follow the exact
  method);
* on a larger mesh the returned iterate's nonlinear residual, recomputed by the
  oracle on sampled cells from the returned velocity, is the one the library
  reports as converged.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mass as omass  # noqa: E402
from oracle import nonlinear  # noqa: E402
from oracle.mesh import BoxMesh  # noqa: E402
from oracle.sipg import SIPG  # noqa: E402
from paper_2506_14424_gb300 import Context, SipgError, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f64ff": 1e-13, "f32": 2e-6}


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("dims,k,op", [((5, 4, 3), 2, "viscous"), ((7, 3, 3), 3, "viscous"),
                                       ((6, 5, 3), 2, "poisson"), ((3, 3, 2), 5, "viscous")])
@pytest.mark.parametrize("arith", ["f64", "f64ff", "f32"])
@pytest.mark.parametrize("inverse", [False, True])
def test_mass_matches_oracle(dims, k, op, arith, inverse):
    ext = (1.0, 0.8, 0.6)
    ctx = Context(*dims, k, extent=ext)
    kk = k if op == "viscous" else k - 1
    S = SIPG(BoxMesh(*dims, extent=ext), kk, 3 if op == "viscous" else 1)
    x = inputs.uniform_vector(S.n_dofs, seed=11)
    coeff = 3.5
    ref = omass.apply_inverse_mass(S, x, coeff) if inverse else omass.apply_mass(S, x, coeff)
    dt = torch.float32 if arith == "f32" else torch.float64
    xd = torch.tensor(x, dtype=dt, device="cuda")
    y = ctx.mass(op, xd, coeff=coeff, arith=arith, inverse=inverse)
    assert _rel(y.double().cpu().numpy(), ref) <= TOL[arith]
    ctx.mass(op, xd, xd, coeff=coeff, arith=arith, inverse=inverse)  # in place
    assert torch.equal(xd, y)
    ctx.close()


def test_mass_full_size_sampled_cells_and_round_trip():
    N, k = 32, 3
    ctx = Context(N, N, N, k)
    n = ctx.n_dofs("viscous")
    x = torch.tensor(inputs.uniform_vector(n, seed=12), device="cuda")
    y = ctx.mass("viscous", x, coeff=2.0, arith="f64ff")
    z = ctx.mass("viscous", y, coeff=2.0, arith="f64ff", inverse=True)
    assert _rel(z.cpu().numpy(), x.cpu().numpy()) <= 1e-13
    Me = 2.0 * omass.mass_block(SIPG(BoxMesh(N, N, N), k, 3))
    m = Me.shape[0]
    xh, yh = x.cpu().numpy().reshape(-1, m), y.cpu().numpy().reshape(-1, m)
    for e in [0, 1, N * N * N // 2 + 7, N * N * N - 1]:
        assert _rel(yh[e], Me @ xh[e]) <= 1e-13
    ctx.close()


def test_mass_rejects_bad_arguments():
    ctx = Context(2, 2, 2, 2)
    x = torch.zeros(ctx.n_dofs("viscous"), dtype=torch.float64, device="cuda")
    with pytest.raises(SipgError):
        ctx.mass("viscous", x, coeff=0.0, inverse=True)
    ctx.close()


def _picard_case(dims=(2, 2, 2), k=2, m=10.0, amp=1.0):
    S = SIPG(BoxMesh(*dims), k, 3)
    modes = inputs.fourier_modes(3)
    uh = S.interpolate(lambda x: amp * inputs.fourier_field(x, modes))
    return S, uh, omass.apply_mass(S, uh, m), m


@pytest.mark.parametrize("aitken", [True, False])
def test_picard_iterates_match_oracle(aitken):
    S, uh, b, m = _picard_case()
    rh = inputs.carreau_blood_like()
    ref = nonlinear.viscous_step_picard(S, rh, b, uh, m, rtol=1e-9, maxit=30, aitken=aitken)
    assert ref['converged']
    ctx = Context(2, 2, 2, 2)
    bd = torch.tensor(b, device="cuda")
    ud = torch.tensor(uh, device="cuda")
    out = ctx.picard_solve(rh, bd, ud, mass=m, rtol=1e-9, atol=0.0, maxit=30, aitken=aitken,
                           lin_rtol=1e-13, lin_atol=1e-13 * np.linalg.norm(b), lin_maxit=1000)
    assert out['status'] == 0
    assert out['iterations'] == ref['iterations']
    res_ref = np.array(ref['residuals'])
    res = np.array(out['residuals'])
    keep = res_ref > 1e-7 * res_ref[0]
    assert np.allclose(res[keep], res_ref[keep], rtol=1e-6)
    assert np.allclose(out['omegas'], ref['omegas'], rtol=1e-6)
    assert _rel(ud.cpu().numpy(), ref['u']) <= 1e-9
    # the stored viscosity is that of the returned iterate
    nc, nf = ctx.get_viscosity(0)
    ref_nc, ref_nf = S.viscosity_at_points(rh, ud.cpu().numpy())
    assert _rel(nc.cpu().numpy(), ref_nc) <= 1e-13
    ctx.close()


def test_picard_larger_mesh_residual_on_sampled_cells():
    dims, k, m = (8, 8, 8), 3, 20.0
    S = SIPG(BoxMesh(*dims), k, 3)
    ctx = Context(*dims, k, krylov_arith="f64ff")
    pts = ctx.node_points("viscous", 0)
    modes = inputs.fourier_modes(3)
    n3 = (k + 1) ** 3
    vals = inputs.fourier_field(pts.reshape(-1, 3), modes).reshape(-1, n3, 3)
    uh = torch.tensor(np.ascontiguousarray(vals.transpose(0, 2, 1)).reshape(-1), device="cuda")
    b = ctx.mass("viscous", uh, coeff=m, arith="f64ff")
    u = uh.clone()
    rh = inputs.carreau_blood_like()
    out = ctx.picard_solve(rh, b, u, mass=m, rtol=1e-8, maxit=40, lin_rtol=1e-4)
    assert out['status'] == 0 and out['res'] <= 1e-8 * out['res0']
    assert out['omegas'][0] == 1.0
    uhost, bhost = u.cpu().numpy(), b.cpu().numpy()
    C = S.mesh.n_cells
    mb = S.n_dofs_cell
    for e in [0, 77, C // 2 + 3, C - 1]:
        nbh = [e] + [S.mesh.neighbor(e, f) for f in range(6) if S.mesh.boundary_type(e, f) == 'I']
        nc, nf = S.viscosity_at_points(rh, uhost, cells=nbh)
        r_e = bhost[e * mb:(e + 1) * mb] - S.apply(uhost, nc, nf, mass=m, cells=[e])[0]
        assert np.linalg.norm(r_e) <= 1.05 * out['res'] + 1e-12 * np.linalg.norm(bhost)
    ctx.close()
