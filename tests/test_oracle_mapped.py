"""Pins for the oracle's SIPG operators on trilinear cells (no GPU).

* without jitter the element blocks equal the affine box oracle's (which has
  its own pins), viscous and Poisson, with a mass term;
* on a jittered mesh: symmetry; the all-Neumann viscous operator annihilates the
  six rigid-body modes a + b x x (linear in x: represented exactly on
  trilinear cells, eps = 0 and no jumps) - this pins J^-1, the normals and the
  surface weights; the all-Neumann Poisson operator annihilates constants;
  Dirichlet operators are positive definite;
* geometry: cell volumes add up to the box; every cell surface is closed,
  sum over its faces of n dA = 0.
"""
import numpy as np
import pytest

from oracle.mapped import MappedMesh, MappedSIPG, box_vertices, jittered_vertices
from oracle.mesh import BoxMesh
from oracle.sipg import SIPG

RH = {'law': 'analytic'}


@pytest.mark.parametrize("ncomp,k", [(3, 2), (1, 3)])
def test_unjittered_equals_affine(ncomp, k):
    dims, ext = (2, 2, 1), (1.0, 0.8, 0.5)
    box = BoxMesh(*dims, extent=ext, bc=('D', 'N', 'D', 'D', 'N', 'D'))
    mm = MappedMesh(*dims, box_vertices(*dims, ext), bc=box.bc)
    A, B = SIPG(box, k, ncomp), MappedSIPG(mm, k, ncomp)
    if ncomp == 3:
        nc, nf = A.viscosity_at_points(RH)
        nc2, nf2 = B.viscosity_at_points(RH)
        assert np.abs(nc - nc2).max() <= 1e-14 and np.abs(nf - nf2).max() <= 1e-14
        Ma, Mb = A.assemble(nc, nf, mass=2.0).toarray(), B.assemble(nc, nf, mass=2.0).toarray()
    else:
        Ma, Mb = A.assemble(mass=2.0).toarray(), B.assemble(mass=2.0).toarray()
    assert np.abs(Ma - Mb).max() <= 1e-12 * np.abs(Ma).max()


def _jittered(dims, bc, amp=0.15, seed=4):
    return MappedMesh(*dims, jittered_vertices(*dims, amp=amp, seed=seed), bc=bc)


def test_geometry_closed_cells_and_volume():
    mm = _jittered((3, 2, 2), ('D',) * 6)
    S = MappedSIPG(mm, 2, 1)
    vol = 0.0
    for e in range(mm.n_cells):
        vol += S.volume(e)
        tot = np.zeros(3)
        for f in range(6):
            _, _, n, W = S.face_geometry(e, f)
            tot += W @ n
        assert np.abs(tot).max() <= 1e-13
    assert abs(vol - 1.0) <= 1e-13


@pytest.mark.parametrize("ncomp,k", [(3, 2), (1, 3)])
def test_jittered_symmetric_and_definite(ncomp, k):
    mm = _jittered((3, 3, 2), ('D',) * 6)
    S = MappedSIPG(mm, k, ncomp)
    if ncomp == 3:
        A = S.assemble(*S.viscosity_at_points(RH)).toarray()
    else:
        A = S.assemble().toarray()
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


def test_jittered_null_spaces():
    mm = _jittered((3, 3, 2), ('N',) * 6)
    S = MappedSIPG(mm, 2, 3)
    A = S.assemble(*S.viscosity_at_points(RH)).toarray()
    modes = [lambda x, c=c: np.eye(3)[c][None, :].repeat(len(x), 0) for c in range(3)]
    for b in np.eye(3):
        modes.append(lambda x, b=b: np.cross(b, x))
    for m in modes:
        r = S.interpolate(m)
        assert np.abs(A @ r).max() <= 1e-12 * np.abs(A).max() * np.abs(r).max()
    P = MappedSIPG(mm, 3, 1)
    Ap = P.assemble().toarray()
    assert np.abs(Ap @ np.ones(P.n_dofs)).max() <= 1e-12 * np.abs(Ap).max()
