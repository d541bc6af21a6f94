"""The C-ABI library loads and exports every symbol include/sipg.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sipg.h")).read()
    return sorted(set(re.findall(r"\b(sipg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_14424_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    from paper_2506_14424_gb300 import _lib
    decl = _declared()
    assert set(decl) == set(_lib.EXPORTS), (set(decl) ^ set(_lib.EXPORTS))
    for name in decl:
        assert hasattr(lib, name), name


def test_default_opts(lib):
    from paper_2506_14424_gb300 import _lib
    o = _lib.Opts()
    lib.sipg_default_opts(ctypes.byref(o))
    assert o.k_u == 3 and o.cheb_degree == 3 and o.cheb_range == 20.0 and o.coarse_max_dofs == 2000
    assert abs(o.cheb_lmax_factor - 1.2) < 1e-15 and o.mg_precision == 1
    assert o.mg_cph == _lib.MG_AUTO and o.mg_setup_lag == 0


@pytest.mark.parametrize("field,value", [("nx", 0), ("k_u", 1), ("k_u", 6), ("bc", 7)])
def test_create_rejects_bad_arguments(lib, field, value):
    """Validation happens before any CUDA call, so this runs without a GPU."""
    from paper_2506_14424_gb300 import _lib
    m = _lib.MeshDesc()
    m.nx = m.ny = m.nz = 2
    m.lx = m.ly = m.lz = 1.0
    o = _lib.Opts()
    lib.sipg_default_opts(ctypes.byref(o))
    if field == "nx":
        m.nx = value
    elif field == "k_u":
        o.k_u = value
    else:
        m.bc_velocity[2] = value
    h = ctypes.c_void_p()
    assert lib.sipg_create(ctypes.byref(m), ctypes.byref(o), None, ctypes.byref(h)) == -1
    assert not h.value


def test_null_arguments(lib):
    assert lib.sipg_create(None, None, None, None) == -1
    assert lib.sipg_destroy(None) == -1


def test_server_rejects_bad_options(lib):
    from paper_2506_14424_gb300 import _lib
    o = _lib.ServerOpts(0, 4, 1, 3)           # zero budget
    h = ctypes.c_void_p()
    assert lib.sipg_server_create(ctypes.byref(o), ctypes.byref(h)) == -1
    o = _lib.ServerOpts(1 << 30, 0, 1, 3)     # no slots
    assert lib.sipg_server_create(ctypes.byref(o), ctypes.byref(h)) == -1


def test_estimate_bytes_grows_with_the_mesh(lib):
    """Size accounting runs without a device (dry run of the hierarchy)."""
    from paper_2506_14424_gb300 import _lib
    vals = []
    for n in (4, 8, 16):
        m = _lib.MeshDesc()
        m.nx = m.ny = m.nz = n
        m.lx = m.ly = m.lz = 1.0
        for i in range(6):
            m.bc_pressure[i] = 1
        o = _lib.Opts()
        lib.sipg_default_opts(ctypes.byref(o))
        b = ctypes.c_int64()
        assert lib.sipg_estimate_bytes(ctypes.byref(m), ctypes.byref(o), ctypes.byref(b)) == 0
        vals.append(b.value)
    # at least the level-0 velocity vectors: 8^3 cells, k=3, 192 DoFs per cell
    assert vals[0] < vals[1] < vals[2] and vals[1] > 8 ** 3 * 192 * 8 * 10
