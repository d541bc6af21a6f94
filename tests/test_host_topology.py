"""Host logic of the grid topology (no GPU): the tables the kernels read for grids with
removed cells and periodic directions, and the masked coarsening of the multigrid
hierarchy, computed by the C library's host code, equal the oracle's mesh.

* neighbour of every face (periodic wrap, removed cells), boundary id and
  boundary-face number of every boundary face, the boundary-face list;
* coarsened active flags, and the refusal when a 2x2x2 block mixes active and
  removed cells;
* the dry run of the hierarchy allocation (sipg_estimate_bytes) on the
  133,120-cell channel grid;
* the multigrid level sequence of a dry hierarchy build (sipg_level_plan) equals
  the oracle's level sequence (p-levels, masked h-coarsening, periodic minimum,
  coarse-size threshold) for the channel, a box and a periodic grid;
* the default hierarchy choice (SIPG_MG_AUTO): the cph levels (the DG level, then the
  continuous twin of every DG level) on a plain box, the DG levels on a grid with
  removed cells or a periodic direction;
* the estimate of trilinear cells counts the stored metric of every level.
"""
import ctypes

import numpy as np
import pytest

from oracle.mesh import BoxMesh
from paper_2506_14424_gb300 import inputs


@pytest.fixture(scope="module")
def lib():
    from paper_2506_14424_gb300 import build, _lib
    build.build()
    return _lib.load()


def _tables(lib, dims, active, periodic):
    act = None if active is None else np.ascontiguousarray(np.asarray(active, dtype=np.uint8).reshape(-1))
    ap = None if act is None else act.ctypes.data_as(ctypes.c_void_p)
    per = (ctypes.c_int * 3)(*[int(bool(p)) for p in periodic])
    nc, nb = ctypes.c_int(), ctypes.c_int()
    assert lib.sipg_topology_tables(*dims, ap, per, ctypes.byref(nc), ctypes.byref(nb), None, None) == 0
    nbr = np.zeros(6 * nc.value, dtype=np.int32)
    bface = np.zeros(max(nb.value, 1), dtype=np.int32)
    assert lib.sipg_topology_tables(*dims, ap, per, ctypes.byref(nc), ctypes.byref(nb),
                                    nbr.ctypes.data_as(ctypes.c_void_p), bface.ctypes.data_as(ctypes.c_void_p)) == 0
    return nc.value, nb.value, nbr, bface[:nb.value]


CASES = [
    ("channel m=2", lambda: inputs.bfs_channel(2, inlet_length=1.0, outlet_length=3.0, depth=1.0)),
    ("channel m=4", lambda: inputs.bfs_channel(4, inlet_length=1.0, outlet_length=3.0, depth=1.0)),
    ("periodic box", lambda: {"dims": (3, 4, 2), "extent": (1.0, 1.0, 1.0), "lo": (0.0, 0.0, 0.0), "active": None,
                              "periodic": (True, False, True)}),
    ("holes", lambda: {"dims": (4, 3, 3), "extent": (1.0, 1.0, 1.0), "lo": (0.0, 0.0, 0.0),
                       "active": np.random.default_rng(5).uniform(size=(3, 3, 4)) > 0.3,
                       "periodic": (False, True, False)}),
]


@pytest.mark.parametrize("name,make", CASES)
def test_topology_tables_match_oracle(lib, name, make):
    c = make()
    mesh = BoxMesh(*c["dims"], extent=c["extent"], lo=c["lo"], active=c["active"], periodic=c["periodic"])
    ncells, nbf, nbr, bface = _tables(lib, c["dims"], c["active"], c["periodic"])
    assert ncells == mesh.n_cells
    faces = mesh.boundary_faces()
    assert nbf == len(faces)
    assert list(bface) == [e * 6 + f for e, f in faces]
    number = {ef: i for i, ef in enumerate(faces)}
    for e in range(mesh.n_cells):
        for f in range(6):
            v = int(nbr[e * 6 + f])
            nb = mesh.neighbor(e, f)
            if nb is not None:
                assert v == nb, (e, f)
            else:
                w = -1 - v
                assert v < 0 and (w & 7) == mesh.boundary_id(e, f) and (w >> 3) == number[(e, f)], (e, f)


def test_coarsen_mask_matches_oracle(lib):
    c = inputs.bfs_channel(4, inlet_length=1.0, outlet_length=3.0, depth=1.0)
    fine = np.ascontiguousarray(c["active"].astype(np.uint8).reshape(-1))
    nx, ny, nz = c["dims"]
    out = np.zeros(fine.size // 8, dtype=np.uint8)
    assert lib.sipg_coarsen_mask(nx, ny, nz, fine.ctypes.data_as(ctypes.c_void_p),
                                 out.ctypes.data_as(ctypes.c_void_p)) == 1
    ref = BoxMesh(*c["dims"], extent=c["extent"], lo=c["lo"], active=c["active"], periodic=c["periodic"]).coarsen()
    assert np.array_equal(out.astype(bool), ref.active)
    bad = fine.copy()
    bad[0] = 1 - bad[0]   # one cell of a block flipped
    assert lib.sipg_coarsen_mask(nx, ny, nz, bad.ctypes.data_as(ctypes.c_void_p),
                                 out.ctypes.data_as(ctypes.c_void_p)) == 0


def test_estimate_bytes_of_the_channel(lib):
    from paper_2506_14424_gb300 import _lib
    c = inputs.bfs_channel(8)
    m = _lib.MeshDesc()
    m.nx, m.ny, m.nz = c["dims"]
    m.lx, m.ly, m.lz = c["extent"]
    for i, b in enumerate("DNDDDD"):
        m.bc_velocity[i] = _lib.BC[b]
    for i, b in enumerate("NDNNNN"):
        m.bc_pressure[i] = _lib.BC[b]
    act = np.ascontiguousarray(c["active"].astype(np.uint8).reshape(-1))
    m.active = act.ctypes.data
    m.bc_removed_velocity, m.bc_removed_pressure = 0, 1
    m.periodic[2] = 1
    for d in range(3):
        m.origin[d] = c["lo"][d]
    o = _lib.Opts()
    lib.sipg_default_opts(ctypes.byref(o))
    o.coarse_max_dofs = 8000
    nbytes = ctypes.c_int64()
    assert lib.sipg_estimate_bytes(ctypes.byref(m), ctypes.byref(o), ctypes.byref(nbytes)) == 0
    n_vel = 133120 * 3 * 64
    # at least the fine-level work vectors; well below the GPU's memory
    assert 10 * 8 * n_vel < nbytes.value < 60e9


def _plan(lib, c, k, op, bc_v="DNDDDD", bc_p="NDNNNN", coarse=2000, mg_cph=0):
    from paper_2506_14424_gb300 import _lib
    m = _lib.MeshDesc()
    m.nx, m.ny, m.nz = c["dims"]
    m.lx, m.ly, m.lz = c["extent"]
    for i in range(6):
        m.bc_velocity[i] = _lib.BC[bc_v[i]]
        m.bc_pressure[i] = _lib.BC[bc_p[i]]
    act = None
    if c["active"] is not None:
        act = np.ascontiguousarray(np.asarray(c["active"], dtype=np.uint8).reshape(-1))
        m.active = act.ctypes.data
    m.bc_removed_velocity, m.bc_removed_pressure = 0, 1
    for d in range(3):
        m.periodic[d] = int(bool(c["periodic"][d]))
        m.origin[d] = c["lo"][d]
    o = _lib.Opts()
    lib.sipg_default_opts(ctypes.byref(o))
    o.k_u = k
    o.coarse_max_dofs = coarse
    o.mg_cph = mg_cph
    nl = ctypes.c_int()
    info = np.zeros(6 * 16, dtype=np.int32)
    assert lib.sipg_level_plan(ctypes.byref(m), ctypes.byref(o), 0 if op == "viscous" else 1, 16,
                               ctypes.byref(nl), info.ctypes.data_as(ctypes.c_void_p)) == 0
    return info[:6 * nl.value].reshape(-1, 6)


@pytest.mark.parametrize("name,make,k,coarse", [
    ("channel m=8", lambda: inputs.bfs_channel(8), 3, 8000),
    ("channel m=4 small", lambda: inputs.bfs_channel(4, inlet_length=1.0, outlet_length=3.0, depth=1.0), 2, 500),
    ("box 16^3", lambda: {"dims": (16, 16, 16), "extent": (1.0, 1.0, 1.0), "lo": (0.0, 0.0, 0.0), "active": None,
                          "periodic": (False, False, False)}, 4, 2000),
    ("periodic 8x4x8", lambda: {"dims": (8, 4, 8), "extent": (1.0, 1.0, 1.0), "lo": (0.0, 0.0, 0.0), "active": None,
                                "periodic": (True, False, True)}, 3, 300),
])
@pytest.mark.parametrize("op", ["viscous", "poisson"])
def test_level_plan_matches_oracle_sequence(lib, name, make, k, coarse, op):
    from oracle import multigrid as omg
    c = make()
    mesh = BoxMesh(*c["dims"], extent=c["extent"], lo=c["lo"], active=c["active"], periodic=c["periodic"])
    ncomp, kk = (3, k) if op == "viscous" else (1, k - 1)
    ref = omg.level_sequence(mesh, kk, ncomp, coarse_threshold=coarse)
    plan = _plan(lib, c, k, op, coarse=coarse)
    assert len(plan) == len(ref)
    for row, (m, kl) in zip(plan, ref):
        assert tuple(row[:3]) == m.n_cells_dir and row[3] == kl and row[4] == m.n_cells
        assert row[5] == m.n_cells * ncomp * (kl + 1) ** 3


def _box(dims, periodic=(False, False, False)):
    return {"dims": dims, "extent": (1.0, 1.0, 1.0), "lo": (0.0, 0.0, 0.0), "active": None, "periodic": periodic}


@pytest.mark.parametrize("op", ["viscous", "poisson"])
def test_default_hierarchy_is_cph_on_plain_boxes(lib, op):
    from paper_2506_14424_gb300 import _lib
    k, coarse = 4, 2000
    ncomp, kk = (3, k) if op == "viscous" else (1, k - 1)
    box = _box((8, 8, 8))
    dg = _plan(lib, box, k, op, coarse=coarse, mg_cph=_lib.MG_DG)
    auto = _plan(lib, box, k, op, coarse=coarse, mg_cph=_lib.MG_AUTO)
    assert np.array_equal(auto, _plan(lib, box, k, op, coarse=coarse, mg_cph=_lib.MG_CPH))
    # [DG level 0, continuous twin of every DG level]: same cells and degree, shared nodes
    assert len(auto) == len(dg) + 1
    assert np.array_equal(auto[0], dg[0])
    for row, d in zip(auto[1:], dg):
        assert np.array_equal(row[:5], d[:5])
        nx, ny, nz, kl = d[0], d[1], d[2], d[3]
        assert row[5] == ncomp * (nx * kl + 1) * (ny * kl + 1) * (nz * kl + 1)
    assert kk == dg[0][3]
    # the continuous levels are built for plain boxes only: auto keeps DG elsewhere
    per = _box((8, 4, 8), periodic=(True, False, True))
    assert np.array_equal(_plan(lib, per, 3, op, coarse=300, mg_cph=_lib.MG_AUTO),
                          _plan(lib, per, 3, op, coarse=300, mg_cph=_lib.MG_DG))
    chan = inputs.bfs_channel(4, inlet_length=1.0, outlet_length=3.0, depth=1.0)
    assert np.array_equal(_plan(lib, chan, 2, op, coarse=500, mg_cph=_lib.MG_AUTO),
                          _plan(lib, chan, 2, op, coarse=500, mg_cph=_lib.MG_DG))


def test_estimate_counts_the_trilinear_metric(lib):
    """Trilinear cells add the stored metric of every level of both hierarchies to the
    estimate: 12 bytes (FP64 + FP32) per value, 10 n^3 cell values (J^-1, w det J) and
    6 x 13 n^2 face values (J^-1, unit normal, surface weight) per cell; they drop the
    float-float split buffer of level 0 (8 bytes per DoF), which only the affine
    float-float operator uses."""
    from oracle.mapped import jittered_vertices
    from paper_2506_14424_gb300 import _lib
    dims, k = (6, 4, 4), 3
    V = np.ascontiguousarray(jittered_vertices(*dims, amp=0.05, seed=1), dtype=np.float64)
    est = []
    for verts in (None, V):
        m = _lib.MeshDesc()
        m.nx, m.ny, m.nz = dims
        m.lx = m.ly = m.lz = 1.0
        for i in range(6):
            m.bc_velocity[i] = _lib.BC["D"]
            m.bc_pressure[i] = _lib.BC["N"]
        if verts is not None:
            m.vertices = verts.ctypes.data
        o = _lib.Opts()
        lib.sipg_default_opts(ctypes.byref(o))
        o.k_u = k
        o.mg_cph = _lib.MG_DG
        nbytes = ctypes.c_int64()
        assert lib.sipg_estimate_bytes(ctypes.byref(m), ctypes.byref(o), ctypes.byref(nbytes)) == 0
        est.append(nbytes.value)
    box = _box(dims)
    metric = split = 0
    for op in ("viscous", "poisson"):
        plan = _plan(lib, box, k, op, bc_v="DDDDDD", bc_p="NNNNNN", coarse=2000, mg_cph=_lib.MG_DG)
        for row in plan:
            n = int(row[3]) + 1
            metric += 12 * int(row[4]) * (10 * n ** 3 + 78 * n ** 2)
        split += 8 * int(plan[0][5])
    assert est[1] - est[0] == metric - split
