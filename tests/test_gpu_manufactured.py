"""GPU parity of the manufactured-solution loads (sipg_rhs_manufactured) against the
oracle's over-integrated load vectors, and the 4^3, k = 2 manufactured solve end to end.

* velocity case (u = s(x) (1, -1, 2), analytic viscosity) and pressure case
  (p = cos cos cos, -lap p = 3 pi^2 p), degrees 2..5, boxes of unequal sides;
* the viscous MG-CG solve of the 4^3-cell, k = 2 problem from the GPU load
  reaches the oracle's sparse-LU solution, whose L2 error against u the oracle's
  convergence pin bounds.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")

from oracle import manufactured as mms  # noqa: E402
from oracle.mesh import BoxMesh  # noqa: E402
from oracle.sipg import SIPG  # noqa: E402
from paper_2506_14424_gb300 import Context  # noqa: E402

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("dims,k,ext", [((4, 4, 4), 2, (1.0, 1.0, 1.0)), ((3, 2, 5), 3, (1.0, 0.7, 1.2)),
                                        ((2, 2, 2), 5, (1.0, 1.0, 1.0)), ((2, 3, 1), 4, (0.5, 1.0, 1.0))])
def test_manufactured_loads_match_oracle(dims, k, ext):
    mesh = BoxMesh(*dims, extent=ext)
    ctx = Context(*dims, k, extent=ext)
    S = SIPG(mesh, k, 3)
    ref = mms.load_vector(S, mms.velocity_force)
    assert _rel(ctx.rhs_manufactured("velocity").cpu().numpy(), ref) <= 1e-12
    P = SIPG(mesh.with_bc(('N',) * 6), k - 1, 1)
    ref = mms.load_vector(P, mms.pressure_force)
    assert _rel(ctx.rhs_manufactured("pressure").cpu().numpy(), ref) <= 1e-12
    ctx.close()


def test_4cubed_k2_manufactured_solve():
    dims, k = (4, 4, 4), 2
    ctx = Context(*dims, k)
    ctx.set_viscosity({'law': 'analytic'})
    b = ctx.rhs_manufactured("velocity")
    x, st = ctx.solve("viscous", b, rtol=1e-12, maxit=500, precond="mg")
    S = SIPG(BoxMesh(*dims), k, 3)
    A = S.assemble(*S.viscosity_at_points({'law': 'analytic'}))
    ref = spla.spsolve(A.tocsc(), mms.load_vector(S, mms.velocity_force))
    assert _rel(x.cpu().numpy(), ref) <= 1e-9
    err = mms.l2_error(S, x.cpu().numpy(), mms.velocity_exact)
    assert err <= 1.01 * mms.l2_error(S, ref, mms.velocity_exact)
    ctx.close()
