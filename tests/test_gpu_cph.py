"""GPU parity of the continuous ("cph") multigrid levels (Sec. 5.4) against the oracle.

* the hierarchy is [DG level 0, continuous twins of the DG sequence];
* transfers (DG -> continuous injection and its transpose, composed
  continuous prolongations and restrictions) equal the oracle's matrices;
* the diagonal of every continuous level equals that of P^T A_DG P;
* an FP64 V-cycle equals the oracle's V-cycle on the oracle's cph matrices
  (viscous with Dirichlet walls, all-Neumann Poisson with the regularised
  coarse solve);
* MG-CG with the cph hierarchy (FP32 V-cycle) solves a high-contrast sinker
  problem to the oracle's residual bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cph  # noqa: E402
from oracle import multigrid as omg  # noqa: E402
from oracle.mesh import BoxMesh  # noqa: E402
from oracle.sipg import SIPG  # noqa: E402
from paper_2506_14424_gb300 import Context, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _dev(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def _oracle_cph(dims, k, op, rheo, bc, coarse):
    ncomp = 3 if op == "viscous" else 1
    kk = k if op == "viscous" else k - 1
    mesh = BoxMesh(*dims, bc=tuple(bc))
    levels = omg.level_sequence(mesh, kk, ncomp, coarse_threshold=coarse)
    if op == "viscous":
        nus = omg.level_viscosity(levels, rheo, None)
        dg = [SIPG(m, kl, 3).assemble(*nus[j]) for j, (m, kl) in enumerate(levels)]
    else:
        dg = [SIPG(m, kl, 1).assemble() for m, kl in levels]
    return levels, cph.cph_levels(levels, dg, ncomp)


@pytest.mark.parametrize("op,bc", [("viscous", "DDDDDD"), ("poisson", "NNNNNN")])
def test_cph_transfers_and_diagonals(op, bc):
    dims, k = (4, 2, 2), 4
    kw = {"bc_velocity": bc} if op == "viscous" else {"bc_pressure": bc}
    ctx = Context(*dims, k, coarse_max_dofs=100, mg_cph=True, mg_precision="f64", **kw)
    rheo = {'law': 'analytic'}
    ctx.set_viscosity(rheo)
    levels, (mats, pro) = _oracle_cph(dims, k, op, rheo, bc, 100)
    assert ctx.num_levels(op) == len(mats) == len(levels) + 1
    for level, P in enumerate(pro):
        xc = inputs.uniform_vector(P.shape[1], seed=30 + level)
        xf = inputs.uniform_vector(P.shape[0], seed=40 + level)
        assert _rel(ctx.transfer(op, level, +1, _dev(xc)).cpu().numpy(), P @ xc) <= 1e-13
        assert _rel(ctx.transfer(op, level, -1, _dev(xf)).cpu().numpy(), P.T @ xf) <= 1e-13
        y32 = ctx.transfer(op, level, -1, _dev(xf, torch.float32)).double().cpu().numpy()
        assert _rel(y32, P.T @ xf) <= 1e-6
    if op == "poisson":  # the Poisson levels are set up on first use
        ctx.vcycle(op, _dev(np.zeros(mats[0].shape[0])))
    for level in range(len(mats)):
        got = ctx.inverse_diagonal(op, level).cpu().numpy()
        assert _rel(got, 1.0 / mats[level].diagonal()) <= 1e-12, level
    ctx.close()


@pytest.mark.parametrize("op,bc", [("viscous", "DDDDDD"), ("poisson", "NNNNNN")])
def test_cph_vcycle_f64_matches_oracle(op, bc):
    dims, k = (4, 4, 4), 3
    kw = {"bc_velocity": bc} if op == "viscous" else {"bc_pressure": bc}
    ctx = Context(*dims, k, mg_precision="f64", coarse_max_dofs=300, mg_cph=True, **kw)
    rheo = {'law': 'analytic'}
    ctx.set_viscosity(rheo)
    _, (mats, pro) = _oracle_cph(dims, k, op, rheo, bc, 300)
    b = inputs.uniform_vector(mats[0].shape[0], seed=70)
    if op == "poisson":
        b -= b.mean()
    x = ctx.vcycle(op, _dev(b)).cpu().numpy()  # sets the levels up first
    lmax = [1.2 * ctx.lmax_estimate(op, level) for level in range(len(mats) - 1)]
    coarse = mats[-1].toarray()
    if op == "poisson":
        coarse = coarse + np.mean(np.diag(coarse)) / coarse.shape[0]
    V = omg.VCycle(mats, pro, 3, lmax)
    V.coarse = coarse
    ref = V(b)
    if op == "poisson":
        ref -= ref.mean()
        x -= x.mean()
    assert _rel(x, ref) <= 1e-10
    ctx.close()


@pytest.mark.parametrize("cph_on", [True, False])
def test_cph_mg_cg_solve(cph_on):
    dims, k = (4, 4, 2), 3
    rheo = inputs.sinker(seed=2, count=8, radius=0.2, nu_max=1e4)
    ctx = Context(*dims, k, coarse_max_dofs=300, mg_cph=cph_on)
    ctx.set_viscosity(rheo)
    S = SIPG(BoxMesh(*dims), k, 3)
    A = S.assemble(*S.viscosity_at_points(rheo))
    u_star = inputs.uniform_vector(S.n_dofs, seed=80)
    b = A @ u_star
    x, st = ctx.solve("viscous", _dev(b), rtol=1e-8, precond="mg", maxit=300)
    xg = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xg) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(b)
    assert st["iterations"] < 80, st
    ctx.close()
