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
