"""GPU parity of the SIPG operators on trilinear cells (jittered meshes) against the oracle.

* viscous applies (constant, analytic, Carreau-Yasuda viscosity; Dirichlet and
  mixed walls) and Poisson applies equal the oracle's per-point-geometry blocks,
  degrees 1..5, meshes of several cells per direction;
* the stored viscosity equals the oracle's at every cell and face point;
* without jitter the trilinear kernel equals the affine kernel;
* an unpreconditioned CG solve reaches the oracle's sparse-LU solution;
* the operator diagonal (Jacobi inside the Chebyshev smoother) equals the
  oracle's assembled diagonal; the FP64 hp-multigrid on trilinear levels
  (h-levels from every other vertex) preconditions CG to the oracle's solution
  and cuts the iteration count against Jacobi;
* at 16^3, k = 3 rows of sampled cells equal the oracle's rows;
* the calls built for the box only refuse a trilinear mesh.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")

from oracle.mapped import MappedMesh, MappedSIPG, box_vertices, jittered_vertices  # noqa: E402
from paper_2506_14424_gb300 import Context, SipgError, inputs  # noqa: E402

pytestmark = pytest.mark.gpu

CARREAU = {'law': 'carreau', 'eta0': 1.0, 'eta_inf': 1e-3, 'kappa': 1.0, 'lam': 1.0, 'a': 2.0, 'b': 0.5}


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("dims,k,bc,law", [((3, 2, 2), 3, "DDDDDD", "carreau"), ((2, 3, 2), 2, "DNDDND", "analytic"),
                                           ((2, 2, 2), 5, "DDDDDD", "constant"), ((3, 3, 2), 4, "DDNDDD", "carreau")])
def test_viscous_apply_matches_oracle(dims, k, bc, law):
    V = jittered_vertices(*dims, amp=0.15, seed=4)
    S = MappedSIPG(MappedMesh(*dims, V, bc=tuple(bc)), k, 3)
    rh = {'constant': {'law': 'constant', 'nu': 0.7}, 'analytic': {'law': 'analytic'}, 'carreau': CARREAU}[law]
    u = S.interpolate(lambda x: inputs.fourier_field(x, inputs.fourier_modes(1)))
    nc, nf = S.viscosity_at_points(rh, u)
    x = inputs.uniform_vector(S.n_dofs, 5)
    ref = S.apply(x, nc, nf, mass=1.5)
    ctx = Context(*dims, k, bc_velocity=bc, vertices=V)
    ctx.set_viscosity(rh, _dev(u))
    gnc, gnf = ctx.get_viscosity(0)
    assert _rel(gnc.cpu().numpy(), nc) <= 1e-13 and _rel(gnf.cpu().numpy(), nf) <= 1e-13
    y = ctx.apply("viscous", _dev(x), mass=1.5)
    assert _rel(y.cpu().numpy(), ref) <= 1e-12
    ctx.close()


@pytest.mark.parametrize("dims,k", [((3, 2, 2), 2), ((2, 2, 3), 4)])
def test_poisson_apply_matches_oracle(dims, k):
    V = jittered_vertices(*dims, amp=0.15, seed=6)
    S = MappedSIPG(MappedMesh(*dims, V, bc=('N',) * 6), k - 1, 1)
    x = inputs.uniform_vector(S.n_dofs, 7)
    ref = S.apply(x)
    ctx = Context(*dims, k, vertices=V)
    y = ctx.apply("poisson", _dev(x))
    assert _rel(y.cpu().numpy(), ref) <= 1e-12
    ctx.close()


def test_unjittered_equals_affine_kernel():
    dims, k = (4, 3, 2), 3
    ext = (1.0, 0.75, 0.5)
    box = Context(*dims, k, extent=ext)
    mapped = Context(*dims, k, extent=ext, vertices=box_vertices(*dims, ext))
    u = torch.tensor(inputs.uniform_vector(box.n_dofs("viscous"), 3), device="cuda")
    for c in (box, mapped):
        c.set_viscosity(CARREAU, u)
    x = torch.tensor(inputs.uniform_vector(box.n_dofs("viscous"), 4), device="cuda")
    assert _rel(mapped.apply("viscous", x).cpu().numpy(), box.apply("viscous", x).cpu().numpy()) <= 1e-12
    xp = torch.tensor(inputs.uniform_vector(box.n_dofs("poisson"), 5), device="cuda")
    assert _rel(mapped.apply("poisson", xp).cpu().numpy(), box.apply("poisson", xp).cpu().numpy()) <= 1e-12
    box.close()
    mapped.close()


def test_cg_solve_matches_oracle():
    dims, k, m = (2, 2, 2), 2, 5.0
    V = jittered_vertices(*dims, amp=0.15, seed=8)
    S = MappedSIPG(MappedMesh(*dims, V), k, 3)
    u = S.interpolate(lambda x: inputs.fourier_field(x, inputs.fourier_modes(1)))
    nc, nf = S.viscosity_at_points(CARREAU, u)
    b = inputs.uniform_vector(S.n_dofs, 9)
    ref = spla.spsolve(S.assemble(nc, nf, mass=m).tocsc(), b)
    ctx = Context(*dims, k, vertices=V)
    ctx.set_viscosity(CARREAU, _dev(u))
    x, st = ctx.solve("viscous", _dev(b), rtol=1e-13, maxit=5000, precond="none", mass=m)
    assert _rel(x.cpu().numpy(), ref) <= 1e-9
    ctx.close()


def test_sampled_rows_at_16cubed():
    N, k = 16, 3
    V = jittered_vertices(N, N, N, amp=0.1, seed=10)
    S = MappedSIPG(MappedMesh(N, N, N, V), k, 3)
    ctx = Context(N, N, N, k, vertices=V)
    n = ctx.n_dofs("viscous")
    u = inputs.uniform_vector(n, 11)
    x = inputs.uniform_vector(n, 12)
    ctx.set_viscosity(CARREAU, _dev(u))
    y = ctx.apply("viscous", _dev(x)).cpu().numpy().reshape(N ** 3, -1)
    for e in [0, 1, N * N * N // 2 + 5, N ** 3 - 1]:
        cells = [e] + [S.mesh.neighbor(e, f) for f in range(6) if S.mesh.boundary_type(e, f) == 'I']
        nc, nf = S.viscosity_at_points(CARREAU, u, cells=cells)
        ref = S.rows(x, [e], nc, nf)[0]
        assert _rel(y[e], ref) <= 1e-12
    ctx.close()


@pytest.mark.parametrize("ncomp", [3, 1])
def test_diagonal_matches_oracle(ncomp):
    dims, k = (3, 2, 2), 3
    V = jittered_vertices(*dims, amp=0.15, seed=12)
    bc = ('D', 'D', 'N', 'D', 'D', 'D')
    ctx = Context(*dims, k, vertices=V, bc_velocity="".join(bc), bc_pressure="NNDNNN")
    if ncomp == 3:
        S = MappedSIPG(MappedMesh(*dims, V, bc=bc), k, 3)
        u = S.interpolate(lambda x: inputs.fourier_field(x, inputs.fourier_modes(1)))
        nc, nf = S.viscosity_at_points(CARREAU, u)
        A = S.assemble(nc, nf)
        ctx.set_viscosity(CARREAU, _dev(u))
        got = ctx.inverse_diagonal("viscous", 0).cpu().numpy()
    else:
        S = MappedSIPG(MappedMesh(*dims, V, bc=('N', 'N', 'D', 'N', 'N', 'N')), k - 1, 1)
        A = S.assemble()
        x = torch.zeros(ctx.n_dofs("poisson"), dtype=torch.float64, device="cuda")
        ctx.solve("poisson", x + 1.0, precond="mg", maxit=1, check=False)  # sets up the Poisson levels
        got = ctx.inverse_diagonal("poisson", 0).cpu().numpy()
    assert _rel(got, 1.0 / A.diagonal()) <= 1e-12
    ctx.close()


def test_multigrid_solve_on_jittered_mesh_matches_oracle():
    dims, k, m = (4, 4, 4), 2, 2.0
    V = jittered_vertices(*dims, amp=0.1, seed=14)
    S = MappedSIPG(MappedMesh(*dims, V), k, 3)
    u = S.interpolate(lambda x: inputs.fourier_field(x, inputs.fourier_modes(1)))
    nc, nf = S.viscosity_at_points(CARREAU, u)
    b = inputs.uniform_vector(S.n_dofs, 15)
    ref = spla.spsolve(S.assemble(nc, nf, mass=m).tocsc(), b)
    ctx = Context(*dims, k, vertices=V, coarse_max_dofs=300)
    assert ctx.num_levels("viscous") >= 3  # p-levels and an h-level on the trilinear mesh
    ctx.set_viscosity(CARREAU, _dev(u))
    x, st = ctx.solve("viscous", _dev(b), rtol=1e-12, maxit=200, precond="mg", mass=m)
    assert _rel(x.cpu().numpy(), ref) <= 1e-9
    assert st["iterations"] <= 40, st
    ctx.close()


def test_multigrid_cuts_iterations_at_8cubed():
    N, k = 8, 3
    V = jittered_vertices(N, N, N, amp=0.05, seed=4)
    ctx = Context(N, N, N, k, vertices=V)
    n = ctx.n_dofs("viscous")
    ctx.set_viscosity(CARREAU, torch.tensor(inputs.uniform_vector(n, 16), device="cuda"))
    b = torch.tensor(inputs.uniform_vector(n, 17), device="cuda")
    _, st_mg = ctx.solve("viscous", b, rtol=1e-8, maxit=500, precond="mg")
    _, st_j = ctx.solve("viscous", b, rtol=1e-8, maxit=3000, precond="jacobi")
    assert st_mg["status"] == 0 and st_j["status"] == 0
    assert st_mg["iterations"] * 5 < st_j["iterations"], (st_mg, st_j)
    ctx.close()


def test_box_only_calls_refuse_trilinear_cells():
    """Float-float applies and the affine-only step options are refused on trilinear cells;
    the FP32 level apply (mixed-precision multigrid) matches the oracle to FP32 accuracy."""
    dims = (2, 2, 2)
    V = jittered_vertices(*dims, amp=0.1)
    ctx = Context(*dims, 2, vertices=V)
    x = torch.zeros(ctx.n_dofs("viscous"), dtype=torch.float64, device="cuda")
    ctx.set_viscosity({'law': 'constant', 'nu': 1.0})
    with pytest.raises(SipgError):
        ctx.apply("viscous", x, arith="f64ff")
    ctx.step_init(x)
    for kw in ({"penalty": True}, {"convective_mode": "linear_implicit"}):
        with pytest.raises(SipgError):
            ctx.step({'law': 'constant', 'nu': 1.0}, 0.01, **kw)
    S = MappedSIPG(MappedMesh(*dims, V), 2, 3)
    xr = inputs.uniform_vector(S.n_dofs, seed=3)
    y32 = ctx.apply("viscous", torch.tensor(xr, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    ref = S.apply(xr, *S.viscosity_at_points({'law': 'constant', 'nu': 1.0}))
    assert np.abs(y32 - ref).max() <= 2e-5 * np.abs(ref).max()
    ctx.close()
