"""GPU parity of the multigrid pieces and the CG solve against the oracle.

* transfers: the GPU prolongation/restriction equal the oracle's explicit
  embedding matrices (and their transposes);
* Chebyshev-Jacobi smoother and the whole V-cycle in FP64 mode equal the
  oracle's recurrence on the oracle's own matrices (same eigenvalue bound);
  FP32 mode within single-precision tolerance;
* Lanczos estimate bounded by the exact largest eigenvalue of D^-1 A;
* solves: the oracle recomputes the residual of the GPU solution with its own
  operator; on the small analytic case the GPU solution equals the oracle's
  direct solution to 1e-8;
* status codes for iteration limits and NaN input.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import manufactured, solvers  # noqa: E402
from oracle import multigrid as omg  # noqa: E402
from oracle.mesh import BoxMesh  # noqa: E402
from oracle.sipg import SIPG  # noqa: E402
from paper_2506_14424_gb300 import Context, SipgError, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _dev(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def _oracle_hierarchy(ctx, op, rheo, bc, mass=0.0, u=None):
    mats, Ps, discs = [], [], []
    levels = []
    for level in range(ctx.num_levels(op)):
        (nx, ny, nz), k, _ = ctx.level_info(op, level)
        levels.append((BoxMesh(nx, ny, nz, bc=tuple(bc)), k))
    nus = omg.level_viscosity(levels, rheo, u) if op == "viscous" else None
    for level, (mesh, k) in enumerate(levels):
        if op == "viscous":
            S = SIPG(mesh, k, 3)
            mats.append(S.assemble(*nus[level], mass=mass))
        else:
            S = SIPG(mesh, k, 1)
            mats.append(S.assemble(mass=mass))
        discs.append(S)
        if level > 0:
            F = discs[level - 1]
            nc = 3 if op == "viscous" else 1
            if F.mesh.n_cells == mesh.n_cells:
                Ps.append(omg.prolongation_p(mesh, F.k, k, nc))
            else:
                Ps.append(omg.prolongation_h(F.mesh, mesh, k, nc))
    return mats, Ps, discs


@pytest.mark.parametrize("op", ["viscous", "poisson"])
def test_transfers_match_oracle(op):
    ctx = Context(4, 2, 2, 4, coarse_max_dofs=100, mg_cph=False)
    rheo = {'law': 'analytic'}
    ctx.set_viscosity(rheo)
    _, Ps, _ = _oracle_hierarchy(ctx, op, rheo, "DDDDDD" if op == "viscous" else "NNNNNN")
    for level, P in enumerate(Ps):
        xc = inputs.uniform_vector(P.shape[1], seed=30 + level)
        xf = inputs.uniform_vector(P.shape[0], seed=40 + level)
        assert _rel(ctx.transfer(op, level, +1, _dev(xc)).cpu().numpy(), P @ xc) <= 1e-14
        assert _rel(ctx.transfer(op, level, -1, _dev(xf)).cpu().numpy(), P.T @ xf) <= 1e-14
        y32 = ctx.transfer(op, level, -1, _dev(xf, torch.float32)).double().cpu().numpy()
        assert _rel(y32, P.T @ xf) <= 1e-6


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 2e-5)])
def test_smoother_matches_oracle_chebyshev(prec, tol):
    ctx = Context(3, 3, 2, 3, mg_precision=prec, mg_cph=False)
    rheo = {'law': 'analytic'}
    ctx.set_viscosity(rheo)
    mats, _, _ = _oracle_hierarchy(ctx, "viscous", rheo, "DDDDDD")
    dtype = torch.float64 if prec == "f64" else torch.float32
    for level in range(len(mats) - 1):
        A = mats[level]
        lmax = 1.2 * ctx.lmax_estimate("viscous", level)
        b = inputs.uniform_vector(A.shape[0], seed=50 + level)
        x0 = inputs.uniform_vector(A.shape[0], seed=60 + level)
        x = ctx.smooth("viscous", level, _dev(b, dtype), _dev(x0, dtype)).double().cpu().numpy()
        ref = omg.chebyshev(A, 1.0 / A.diagonal(), b, x0, 3, lmax / 20.0, lmax)
        assert _rel(x, ref) <= tol, level


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 2e-6)])
def test_lanczos_estimate_bounded_by_exact(prec, tol):
    # the estimate is of the operator the smoother applies: FP32 multigrid
    # estimates the FP32-rounded operator (relative perturbation ~ 1e-7)
    ctx = Context(2, 2, 2, 3, mg_precision=prec, mg_cph=False)
    rheo = {'law': 'analytic'}
    ctx.set_viscosity(rheo)
    mats, _, _ = _oracle_hierarchy(ctx, "viscous", rheo, "DDDDDD")
    for level in range(len(mats) - 1):
        A = mats[level].toarray()
        s = 1.0 / np.sqrt(np.diag(A))
        exact = np.linalg.eigvalsh(s[:, None] * A * s[None, :])[-1]
        est = ctx.lmax_estimate("viscous", level)
        assert est <= exact * (1 + tol) and est >= 0.8 * exact, (level, est, exact)


@pytest.mark.parametrize("op,bc", [("viscous", "DDDDDD"), ("poisson", "NNNNNN")])
def test_vcycle_f64_matches_oracle_vcycle(op, bc):
    kw = {"bc_velocity": bc} if op == "viscous" else {"bc_pressure": bc}
    ctx = Context(4, 4, 4, 3, mg_precision="f64", coarse_max_dofs=300, mg_cph=False, **kw)
    rheo = {'law': 'analytic'}
    ctx.set_viscosity(rheo)
    mats, Ps, _ = _oracle_hierarchy(ctx, op, rheo, bc)
    lmax = [1.2 * ctx.lmax_estimate(op, level) for level in range(len(mats) - 1)]
    coarse = mats[-1].toarray()
    if op == "poisson":
        coarse = coarse + np.mean(np.diag(coarse)) / coarse.shape[0]  # same regularised coarse solve
    V = omg.VCycle(mats, Ps, 3, lmax)
    V.coarse = coarse
    b = inputs.uniform_vector(mats[0].shape[0], seed=70)
    if op == "poisson":
        b -= b.mean()
    x = ctx.vcycle(op, _dev(b)).cpu().numpy()
    ref = V(b)
    if op == "poisson":
        ref -= ref.mean()
    assert _rel(x, ref) <= 1e-10


def test_4cubed_k2_jacobi_cg_matches_oracle():
    """4^3 cells, k = 2, analytic viscosity, Dirichlet walls, manufactured load."""
    mesh = BoxMesh(4, 4, 4)
    S = SIPG(mesh, 2, 3)
    rheo = {'law': 'analytic'}
    A = S.assemble(*S.viscosity_at_points(rheo))
    b = manufactured.load_vector(S, manufactured.velocity_force)
    x_ref = solvers.cholesky_solve(A, b)
    ctx = Context(4, 4, 4, 2)
    ctx.set_viscosity(rheo)
    x, st = ctx.solve("viscous", _dev(b), rtol=1e-8, precond="jacobi")
    xg = x.cpu().numpy()
    # (i) the oracle's own residual of the GPU solution
    assert np.linalg.norm(b - A @ xg) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(b)
    assert st["rel_residual"] <= 1e-8
    # (iii) the same discrete solution, tight solve
    x2, _ = ctx.solve("viscous", _dev(b), rtol=1e-13, precond="jacobi", maxit=2000)
    assert np.linalg.norm(x2.cpu().numpy() - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    # the discrete solution approximates the manufactured field like the oracle's
    e_gpu = manufactured.l2_error(S, x2.cpu().numpy(), manufactured.velocity_exact)
    e_ref = manufactured.l2_error(S, x_ref, manufactured.velocity_exact)
    assert abs(e_gpu - e_ref) <= 1e-8 * e_ref


@pytest.mark.parametrize("rheo_name", ["sinker", "carreau"])
def test_level_viscosity_matches_oracle(rheo_name):
    dims, k = (4, 4, 2), 4
    S = SIPG(BoxMesh(*dims), k, 3)
    u = None
    if rheo_name == "sinker":
        rheo = inputs.sinker(seed=2, count=8, radius=0.2, nu_max=1e6)
    else:
        rheo = inputs.carreau_blood_like()
        modes = inputs.fourier_modes(1)
        u = S.interpolate(lambda p: inputs.fourier_field(p, modes))
    ctx = Context(*dims, k, coarse_max_dofs=100, mg_cph=False)
    ctx.set_viscosity(rheo, None if u is None else _dev(u))
    levels = []
    for level in range(ctx.num_levels("viscous")):
        (nx, ny, nz), kl, _ = ctx.level_info("viscous", level)
        levels.append((BoxMesh(nx, ny, nz), kl))
    assert [(m.n_cells, kl) for m, kl in levels] == [(32, 4), (32, 2), (32, 1), (4, 1)]
    for level, (rc, rf) in enumerate(omg.level_viscosity(levels, rheo, u)):
        nc, nf = ctx.get_viscosity(level)
        assert _rel(nc.cpu().numpy(), rc) <= 1e-13, level
        assert _rel(nf.cpu().numpy(), rf) <= 1e-13, level


@pytest.mark.parametrize("hier", ["auto", False])
@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("contrast", [1.0, 1e4, 1e6])
def test_mg_cg_solve_matches_oracle(prec, contrast, hier):
    dims, k = (4, 4, 2), 3
    rheo = inputs.sinker(seed=2, count=8, radius=0.2, nu_max=contrast)
    ctx = Context(*dims, k, mg_precision=prec, coarse_max_dofs=300, mg_cph=hier)
    ctx.set_viscosity(rheo)
    S = SIPG(BoxMesh(*dims), k, 3)
    A = S.assemble(*S.viscosity_at_points(rheo))
    u_star = inputs.uniform_vector(S.n_dofs, seed=80)
    b = A @ u_star
    x, st = ctx.solve("viscous", _dev(b), rtol=1e-8, precond="mg", maxit=200)
    xg = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xg) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(b)
    assert st["iterations"] < 40, st


def test_lagged_multigrid_setup_keeps_the_solution():
    """mg_setup_lag = 3: after a second viscosity update the eigenvalue estimates and the
    coarse inverse of the first are kept (the diagonals follow); the preconditioner is
    still fixed and SPD, so CG reaches the oracle's solution of the new system."""
    dims, k = (4, 4, 2), 3
    ctx = Context(*dims, k, coarse_max_dofs=300, mg_setup_lag=3)
    S = SIPG(BoxMesh(*dims), k, 3)
    its = []
    for contrast in (1e2, 3e2, 1e3):
        rheo = inputs.sinker(seed=2, count=8, radius=0.2, nu_max=contrast)
        ctx.set_viscosity(rheo)
        A = S.assemble(*S.viscosity_at_points(rheo))
        b = A @ inputs.uniform_vector(S.n_dofs, seed=84)
        x, st = ctx.solve("viscous", _dev(b), rtol=1e-8, precond="mg", maxit=300)
        assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(b)
        its.append(st["iterations"])
    assert max(its) < 60, its


def test_poisson_mg_solve_singular():
    dims, kp = (4, 4, 4), 2
    ctx = Context(*dims, kp + 1, coarse_max_dofs=200)
    P = SIPG(BoxMesh(*dims, bc=('N',) * 6), kp, 1)
    A = P.assemble()
    b = manufactured.load_vector(P, lambda x: manufactured.pressure_force(x)[..., None])
    b -= b.mean()
    x, st = ctx.solve("poisson", _dev(b), rtol=1e-8, precond="mg")
    xg = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xg) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(b)
    assert abs(xg.mean()) < 1e-10 * np.abs(xg).max()


def test_krylov_float_float_solve_matches_oracle():
    dims, k = (4, 4, 2), 3
    rheo = inputs.sinker(seed=2, count=8, radius=0.2, nu_max=1e2)
    ctx = Context(*dims, k, coarse_max_dofs=300, krylov_arith="f64ff")
    ctx.set_viscosity(rheo)
    S = SIPG(BoxMesh(*dims), k, 3)
    A = S.assemble(*S.viscosity_at_points(rheo))
    b = A @ inputs.uniform_vector(S.n_dofs, seed=83)
    x, st = ctx.solve("viscous", _dev(b), rtol=1e-10, precond="mg")
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1e-10 * (1 + 1e-6) * np.linalg.norm(b)


def test_viscous_step_operator_mass_solve():
    dims, k = (3, 3, 3), 3
    rheo = {'law': 'analytic'}
    ctx = Context(*dims, k, coarse_max_dofs=400)
    ctx.set_viscosity(rheo)
    S = SIPG(BoxMesh(*dims), k, 3)
    m = 1.5 / 0.01  # gamma0 / dt of BDF2 with dt = 0.01
    A = S.assemble(*S.viscosity_at_points(rheo), mass=m)
    b = A @ inputs.uniform_vector(S.n_dofs, seed=81)
    x, st = ctx.solve("viscous", _dev(b), rtol=1e-10, precond="mg", mass=m)
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1e-10 * (1 + 1e-6) * np.linalg.norm(b)


def test_status_codes():
    ctx = Context(2, 2, 2, 2)
    ctx.set_viscosity({'law': 'analytic'})
    b = _dev(inputs.uniform_vector(ctx.n_dofs(), seed=82))
    _, st = ctx.solve("viscous", b, rtol=1e-14, precond="none", maxit=2, check=False)
    assert st["status"] == -4 and st["iterations"] == 2
    bad = b.clone()
    bad[5] = float("nan")
    with pytest.raises(SipgError) as ei:
        ctx.solve("viscous", bad, precond="jacobi")
    assert ei.value.code == -6
