"""GPU parity of the operator path against the FP64 oracle (through the C ABI).

Tolerance (FP64): ||y_gpu - y_oracle||_inf <= 1e-12 ||y_oracle||_inf; FP32
level operators: 2e-5 (single-precision sum factorisation over O(100) terms).
Meshes are chosen to span several CTAs with a ragged tail (cell counts not a
multiple of the cells-per-CTA of any degree) and both boundary types.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import multigrid as omg  # noqa: E402
from oracle.mesh import BoxMesh  # noqa: E402
from oracle.sipg import SIPG  # noqa: E402
from paper_2506_14424_gb300 import Context, inputs  # noqa: E402

pytestmark = pytest.mark.gpu
TOL64 = 1e-12
TOL32 = 2e-5


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _bc(s):
    return tuple(s)


def _dev(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


CASES = [
    # dims, k, velocity bc, rheology
    ((7, 5, 2), 2, "DDDDDD", {'law': 'analytic'}),           # 70 cells: 3 CTAs of 32, ragged
    ((3, 4, 3), 3, "DNDDND", {'law': 'analytic'}),           # 36 cells: 5 CTAs of 8, ragged
    ((3, 1, 1), 4, "DDDDDD", {'law': 'constant', 'nu': 0.3}),  # 3 cells: 2 CTAs of 2, ragged
    ((1, 1, 3), 5, "NDDNDD", {'law': 'analytic'}),
    ((1, 1, 1), 2, "DDDDDD", {'law': 'analytic'}),
]


@pytest.mark.parametrize("arith", ["f64", "f64ff"])
@pytest.mark.parametrize("dims,k,bc,rheo", CASES)
def test_viscous_apply_f64_matches_oracle(dims, k, bc, rheo, arith):
    ctx = Context(*dims, k, bc_velocity=bc)
    ctx.set_viscosity(rheo)
    S = SIPG(BoxMesh(*dims, bc=_bc(bc)), k, 3)
    nu = S.viscosity_at_points(rheo)
    x = inputs.uniform_vector(S.n_dofs, seed=11)
    y = ctx.apply('viscous', _dev(x), arith=arith).cpu().numpy()
    assert _rel(y, S.apply(x, *nu)) <= TOL64
    # mass term of the viscous-step operator (gamma0/dt) M + A
    y = ctx.apply('viscous', _dev(x), mass=37.5, arith=arith).cpu().numpy()
    assert _rel(y, S.apply(x, *nu, mass=37.5)) <= TOL64


@pytest.mark.parametrize("arith", ["f64", "f64ff"])
@pytest.mark.parametrize("dims,k,bc", [((5, 3, 2), 1, "NNNNNN"), ((3, 2, 4), 2, "DDNNDD"),
                                       ((2, 3, 2), 3, "DDDDDD"), ((2, 2, 2), 4, "NNNNNN")])
def test_poisson_apply_f64_matches_oracle(dims, k, bc, arith):
    ctx = Context(*dims, k + 1, bc_pressure=bc)
    P = SIPG(BoxMesh(*dims, bc=_bc(bc)), k, 1)
    x = inputs.uniform_vector(P.n_dofs, seed=12)
    y = ctx.apply('poisson', _dev(x), arith=arith).cpu().numpy()
    assert _rel(y, P.apply(x)) <= TOL64


@pytest.mark.parametrize("dims,k", [((5, 3, 2), 2), ((3, 2, 3), 3)])
def test_viscous_apply_f32_close_to_oracle(dims, k):
    ctx = Context(*dims, k)
    rheo = {'law': 'analytic'}
    ctx.set_viscosity(rheo)
    S = SIPG(BoxMesh(*dims), k, 3)
    x = inputs.uniform_vector(S.n_dofs, seed=13)
    y = ctx.apply('viscous', _dev(x, torch.float32)).double().cpu().numpy()
    assert _rel(y, S.apply(x, *S.viscosity_at_points(rheo))) <= TOL32


@pytest.mark.parametrize("op", ["viscous", "poisson"])
@pytest.mark.parametrize("dims,k_u", [((7, 3, 2), 3), ((11, 2, 1), 4), ((3, 5, 3), 2)])
def test_f32_level_applies_close_to_oracle(op, dims, k_u):
    """FP32 applies on every p-level of the fine mesh (degrees 1..4 of both
    operators: the register-tiled kernel for degrees 1..3, the shared-memory
    kernel above), anisotropic cells, mixed walls, the mass term; cell counts
    (42, 22, 45) leave ragged warps of 10 and 32 cells."""
    extent = (1.3, 0.7, 2.1)
    bcv, bcp = "DNDDND", "NDNNDN"
    ctx = Context(*dims, k_u, extent=extent, bc_velocity=bcv, bc_pressure=bcp, mg_cph=False)
    rheo = {'law': 'analytic'}
    ctx.set_viscosity(rheo)
    nc = 3 if op == "viscous" else 1
    bc = bcv if op == "viscous" else bcp
    for level in range(ctx.num_levels(op)):
        cells, deg, nd = ctx.level_info(op, level)
        if tuple(cells) != tuple(dims):
            break
        S = SIPG(BoxMesh(*dims, extent=extent, bc=_bc(bc)), deg, nc)
        nu = S.viscosity_at_points(rheo) if nc == 3 else (None, None)
        x = inputs.uniform_vector(S.n_dofs, seed=31 + level)
        for mass in (0.0, 7.5):
            y = ctx.apply(op, _dev(x, torch.float32), mass=mass, level=level).double().cpu().numpy()
            assert _rel(y, S.apply(x, *nu, mass=mass)) <= TOL32, (level, deg, mass)


@pytest.mark.parametrize("rheo_name", ["analytic", "sinker", "carreau"])
def test_viscosity_at_points_matches_oracle(rheo_name):
    dims, k = (4, 3, 3), 3
    mesh = BoxMesh(*dims)
    S = SIPG(mesh, k, 3)
    u = None
    if rheo_name == "analytic":
        rheo = {'law': 'analytic'}
    elif rheo_name == "sinker":
        rheo = inputs.sinker(seed=2, count=8, radius=0.2, nu_max=1e4)
    else:
        rheo = inputs.carreau_blood_like()
        modes = inputs.fourier_modes(1)
        u = S.interpolate(lambda p: inputs.fourier_field(p, modes))
    ctx = Context(*dims, k)
    ctx.set_viscosity(rheo, None if u is None else _dev(u))
    nc, nf = ctx.get_viscosity(0)
    rc, rf = S.viscosity_at_points(rheo, u)
    assert _rel(nc.cpu().numpy(), rc) <= 1e-13
    assert _rel(nf.cpu().numpy(), rf) <= 1e-13
    # and the full viscosity + operator pipeline
    x = inputs.uniform_vector(S.n_dofs, seed=14)
    y = ctx.apply('viscous', _dev(x)).cpu().numpy()
    assert _rel(y, S.apply(x, rc, rf)) <= TOL64


@pytest.mark.parametrize("arith", ["f64", "f64ff"])
def test_apply_is_deterministic(arith):
    ctx = Context(6, 5, 4, 3)
    ctx.set_viscosity({'law': 'analytic'})
    x = _dev(inputs.uniform_vector(ctx.n_dofs(), seed=15))
    y1 = ctx.apply('viscous', x, arith=arith)
    y2 = ctx.apply('viscous', x, arith=arith)
    assert torch.equal(y1, y2)


def test_apply_host_matches_device():
    ctx = Context(3, 3, 2, 3)
    ctx.set_viscosity({'law': 'analytic'})
    x = inputs.uniform_vector(ctx.n_dofs(), seed=16)
    yd = ctx.apply('viscous', _dev(x)).cpu().numpy()
    yh = ctx.apply_host('viscous', x)
    assert np.array_equal(yd, yh)


def test_symmetry_of_gpu_applies():
    ctx = Context(3, 2, 3, 3, bc_velocity="DNDDND")
    ctx.set_viscosity(inputs.sinker(seed=2, count=8, radius=0.3, nu_max=1e3))
    n = ctx.n_dofs()
    x = _dev(inputs.uniform_vector(n, seed=17))
    z = _dev(inputs.uniform_vector(n, seed=18))
    a = torch.dot(z, ctx.apply('viscous', x)).item()
    b = torch.dot(x, ctx.apply('viscous', z)).item()
    assert abs(a - b) <= 1e-12 * abs(a)


def test_full_size_32cubed_sampled_rows():
    """32^3 cells, k = 3, Carreau-Yasuda from the Fourier field: sampled rows."""
    N, k = 32, 3
    mesh = BoxMesh(N, N, N)
    S = SIPG(mesh, k, 3)
    ctx = Context(N, N, N, k)
    modes = inputs.fourier_modes(1)
    pts = ctx.node_points('viscous', 0).reshape(-1, 3)
    u = inputs.fourier_field(pts, modes).reshape(mesh.n_cells, -1, 3).transpose(0, 2, 1).reshape(-1)
    rheo = inputs.carreau_blood_like()
    ctx.set_viscosity(rheo, _dev(u))
    x = inputs.uniform_vector(ctx.n_dofs(), seed=19)
    y = ctx.apply('viscous', _dev(x)).cpu().numpy().reshape(mesh.n_cells, -1)
    yff = ctx.apply('viscous', _dev(x), arith='f64ff').cpu().numpy().reshape(mesh.n_cells, -1)
    # float-float against native FP64 over the whole vector
    assert _rel(yff, y) <= TOL64
    rng = np.random.default_rng(20)
    cells = sorted(set([0, N - 1, N * N * N - 1, (N // 2) * (N * N + N + 1)] +
                       list(rng.integers(0, N ** 3, 12))))
    # the oracle's viscosity on the sampled cells and their neighbours only
    need = set(cells)
    for e in cells:
        for f in range(6):
            nb = mesh.neighbor(e, f)
            if nb is not None:
                need.add(nb)
    nc_ref, nf_ref = S.viscosity_at_points(rheo, u, cells=sorted(need))
    y_ref = S.apply(x, nc_ref, nf_ref, cells=cells)
    assert _rel(y[cells], y_ref) <= TOL64
    assert _rel(yff[cells], y_ref) <= TOL64
    nc, nf = ctx.get_viscosity(0)
    assert _rel(nc.cpu().numpy()[cells], nc_ref[cells]) <= 1e-13
    assert _rel(nf.cpu().numpy()[cells], nf_ref[cells]) <= 1e-13
    # the node coordinates the library reports are the oracle's GLL nodes
    assert np.abs(pts.reshape(mesh.n_cells, -1, 3)[cells[1]] - S.node_points(cells[1])).max() < 1e-15


@pytest.mark.parametrize("op,dims,k", [("viscous", (4, 2, 2), 3), ("poisson", (4, 4, 2), 3)])
def test_inverse_diagonal_matches_oracle(op, dims, k):
    ctx = Context(*dims, k, bc_velocity="DDNDDD", bc_pressure="NNDNNN", mg_cph=False)
    rheo = {'law': 'analytic'}
    ctx.set_viscosity(rheo)
    nlev = ctx.num_levels(op)
    for level in range(nlev):
        (nx, ny, nz), kl, _ = ctx.level_info(op, level)
        mesh = BoxMesh(nx, ny, nz, bc=_bc("DDNDDD" if op == "viscous" else "NNDNNN"))
        if op == "viscous":
            S = SIPG(mesh, kl, 3)
            A = S.assemble(*S.viscosity_at_points(rheo))
        else:
            S = SIPG(mesh, kl, 1)
            A = S.assemble()
        dinv = ctx.inverse_diagonal(op, level).cpu().numpy()
        assert _rel(1.0 / dinv, A.diagonal()) <= TOL64, level


@pytest.mark.parametrize("arith", ["f64", "f64ff"])
def test_anisotropic_cells_and_mixed_walls(arith):
    """Non-cubic box and cells (hx != hy != hz), both operators, mixed boundary types."""
    dims, extent, k = (3, 2, 4), (1.3, 0.7, 2.1), 3
    bcv, bcp = "DNDDND", "NDNNDN"
    ctx = Context(*dims, k, extent=extent, bc_velocity=bcv, bc_pressure=bcp)
    rheo = {'law': 'analytic'}
    ctx.set_viscosity(rheo)
    S = SIPG(BoxMesh(*dims, extent=extent, bc=_bc(bcv)), k, 3)
    x = inputs.uniform_vector(S.n_dofs, seed=21)
    y = ctx.apply('viscous', _dev(x), mass=3.0, arith=arith).cpu().numpy()
    assert _rel(y, S.apply(x, *S.viscosity_at_points(rheo), mass=3.0)) <= TOL64
    P = SIPG(BoxMesh(*dims, extent=extent, bc=_bc(bcp)), k - 1, 1)
    xp = inputs.uniform_vector(P.n_dofs, seed=22)
    yp = ctx.apply('poisson', _dev(xp), arith=arith).cpu().numpy()
    assert _rel(yp, P.apply(xp)) <= TOL64


def test_maximum_size_sampled_rows():
    """48^3 cells, k = 5 (71.7e6 velocity DoFs, the largest served mesh), sphere viscosity."""
    N, k = 48, 5
    mesh = BoxMesh(N, N, N)
    S = SIPG(mesh, k, 3)
    rheo = inputs.sinker(seed=3, count=8, radius=0.1, nu_max=1e2)
    ctx = Context(N, N, N, k)
    ctx.set_viscosity(rheo)
    n = ctx.n_dofs()
    assert n == N ** 3 * 3 * 216
    x = inputs.uniform_vector(n, seed=23)
    xd = _dev(x)
    y = ctx.apply('viscous', xd).cpu().numpy().reshape(mesh.n_cells, -1)
    yff = ctx.apply('viscous', xd, arith='f64ff').cpu().numpy().reshape(mesh.n_cells, -1)
    cells = [0, N * N * N - 1, (N // 2) * (N * N + N + 1) + 7, 12345]
    need = set(cells)
    for e in cells:
        for f in range(6):
            nb = mesh.neighbor(e, f)
            if nb is not None:
                need.add(nb)
    nc, nf = S.viscosity_at_points(rheo, cells=sorted(need))
    y_ref = S.apply(x, nc, nf, cells=cells)
    assert _rel(y[cells], y_ref) <= TOL64
    assert _rel(yff[cells], y_ref) <= TOL64
    ctx.close()
