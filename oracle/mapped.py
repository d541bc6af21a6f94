"""SIPG operators on trilinear (non-affine) hexahedra (oracle, test infrastructure).

Sec. 5 of the paper works on general hexahedral meshes; the box oracle
(``oracle.sipg``) covers affine cells only. Here each cell is the trilinear
image x(xi) = sum_v N_v(xi) X_v of the unit cube through its 8 vertices, as
for the jittered channel mesh of the backward-facing-step workload. The
topology stays structured (cells (i, j, k), neighbours across the six
faces), so two cells that share a face share its four vertices and
parametrise it with the same tangential reference coordinates.

Everything the affine oracle gets from h is computed per quadrature point:
  J = dx/dxi,  W = w_q det J,  grad phi = J^-T grad_xi phi;
  on a face with tangents t1 = dx/dxi_t1, t2 = dx/dxi_t2: the outward unit
  normal n = +-(t1 x t2)/|t1 x t2| and the surface weight w_a w_b |t1 x t2|;
  the penalty factor Lambda_e = sum_f w_f |f| / |Omega_e| with the integrated
  face areas and cell volume (w_f = 1/2 interior, 1 boundary). READING: |f| and
  |Omega_e| are integrated with the operator's own Gauss rule (|t1 x t2| is
  not a polynomial on a trilinear face, so the rule is part of the definition).
The element forms, fluxes, mirror boundary conditions and penalty are those of
``oracle.sipg`` (same readings), with the normal taken per point.

Pins (tests/test_oracle_mapped.py): without jitter the blocks equal the affine
oracle's; with jitter the operators are symmetric, the all-Neumann viscous
operator annihilates the six rigid-body modes (linear in x, hence exactly
represented on trilinear cells) and the Poisson operator the constants, the
Dirichlet operators are positive definite, the cell volumes add up to the box
and every cell surface is closed (sum of n dA = 0).
"""
import numpy as np
import scipy.sparse as sp

from . import basis, quadrature, viscosity
from .mesh import BoxMesh
from .sipg import _sym


class MappedMesh:
    """Structured hexahedral mesh; vertex (i, j, k) at X[k, j, i] (shape (nz+1, ny+1, nx+1, 3)).
    The topology is that of oracle.mesh.BoxMesh: optional removed cells (``active``) and
    periodic directions (the vertices of the first and last layers of a periodic direction
    must then agree up to the period)."""

    def __init__(self, nx, ny, nz, vertices, bc=('D',) * 6, active=None, periodic=(False, False, False)):
        self.topo = BoxMesh(nx, ny, nz, bc=bc, active=active, periodic=periodic)
        self.X = np.asarray(vertices, dtype=np.float64).reshape(nz + 1, ny + 1, nx + 1, 3)
        self.n_cells_dir = (nx, ny, nz)
        self.bc = self.topo.bc

    @property
    def n_cells(self):
        return self.topo.n_cells

    def neighbor(self, e, f):
        return self.topo.neighbor(e, f)

    def boundary_type(self, e, f):
        return self.topo.boundary_type(e, f)

    def boundary_id(self, e, f):
        return self.topo.boundary_id(e, f)

    def boundary_faces(self):
        return self.topo.boundary_faces()

    def cell_ijk(self, e):
        return self.topo.cell_ijk(e)

    def with_bc(self, bc):
        """The same cells and vertices with other boundary types."""
        nx, ny, nz = self.n_cells_dir
        return MappedMesh(nx, ny, nz, self.X, bc=bc, active=self.topo.active, periodic=self.topo.periodic)

    def cell_vertices(self, e):
        """(8, 3), vertex (a, b, c) in {0,1}^3 at index a + 2 b + 4 c."""
        i, j, k = self.topo.cell_ijk(e)
        return np.array([self.X[k + c, j + b, i + a] for c in (0, 1) for b in (0, 1) for a in (0, 1)])


def box_vertices(nx, ny, nz, extent=(1.0, 1.0, 1.0)):
    xs = [np.linspace(0.0, extent[d], n + 1) for d, n in enumerate((nx, ny, nz))]
    Z, Y, Xg = np.meshgrid(xs[2], xs[1], xs[0], indexing='ij')
    return np.stack([Xg, Y, Z], axis=-1)


def jittered_vertices(nx, ny, nz, extent=(1.0, 1.0, 1.0), amp=0.05, seed=4):
    """Box vertices with the interior ones moved by U(-amp h, amp h) per direction
    (h the cell size of that direction); boundary vertices stay, so the walls stay planar."""
    V = box_vertices(nx, ny, nz, extent)
    h = np.array([extent[0] / nx, extent[1] / ny, extent[2] / nz])
    rng = np.random.default_rng(seed)
    J = rng.uniform(-amp, amp, size=V.shape) * h
    J[0, :, :] = J[-1, :, :] = 0.0
    J[:, 0, :] = J[:, -1, :] = 0.0
    J[:, :, 0] = J[:, :, -1] = 0.0
    return V + J


def _trilinear(xi):
    """N (P, 8) and dN/dxi (P, 8, 3) of the trilinear vertex functions."""
    P = xi.shape[0]
    N = np.zeros((P, 8))
    dN = np.zeros((P, 8, 3))
    for c in (0, 1):
        for b in (0, 1):
            for a in (0, 1):
                v = a + 2 * b + 4 * c
                fx = xi[:, 0] if a else 1 - xi[:, 0]
                fy = xi[:, 1] if b else 1 - xi[:, 1]
                fz = xi[:, 2] if c else 1 - xi[:, 2]
                sx, sy, sz = (1.0 if a else -1.0), (1.0 if b else -1.0), (1.0 if c else -1.0)
                N[:, v] = fx * fy * fz
                dN[:, v, 0] = sx * fy * fz
                dN[:, v, 1] = fx * sy * fz
                dN[:, v, 2] = fx * fy * sz
    return N, dN


class MappedSIPG:
    """Explicit element blocks of the viscous (ncomp=3) or Poisson (ncomp=1) operator on trilinear cells."""

    def __init__(self, mesh, k, ncomp, penalty_factor=1.0, face_nu='max', n_quad=None):
        self.mesh = mesh
        self.k = int(k)
        self.n = self.k + 1
        self.nq = int(n_quad) if n_quad is not None else self.n
        self.ncomp = int(ncomp)
        self.C_ip = float(penalty_factor)
        self.face_nu = face_nu
        self.nodes, _ = quadrature.gauss_lobatto(self.n)
        self.gpts, self.gwts = quadrature.gauss_legendre(self.nq)
        n, nq = self.n, self.nq
        self.n_dofs_cell = ncomp * n ** 3
        qz, qy, qx = np.meshgrid(np.arange(nq), np.arange(nq), np.arange(nq), indexing='ij')
        qx, qy, qz = qx.ravel(), qy.ravel(), qz.ravel()
        self.cell_xi = np.stack([self.gpts[qx], self.gpts[qy], self.gpts[qz]], axis=1)
        self.cell_w = self.gwts[qx] * self.gwts[qy] * self.gwts[qz]
        self.cell_phi, self.cell_dphi = basis.tensor_basis(self.nodes, self.cell_xi)
        self.cell_N, self.cell_dN = _trilinear(self.cell_xi)
        self.face_xi, self.face_phi, self.face_dphi, self.face_N, self.face_dN = [], [], [], [], []
        b_idx, a_idx = np.meshgrid(np.arange(nq), np.arange(nq), indexing='ij')
        a_idx, b_idx = a_idx.ravel(), b_idx.ravel()
        self.face_w2 = self.gwts[a_idx] * self.gwts[b_idx]
        for f in range(6):
            d, s = divmod(f, 2)
            t1, t2 = [a for a in range(3) if a != d]
            xi = np.zeros((nq * nq, 3))
            xi[:, d] = float(s)
            xi[:, t1] = self.gpts[a_idx]
            xi[:, t2] = self.gpts[b_idx]
            phi, dphi = basis.tensor_basis(self.nodes, xi)
            Nf, dNf = _trilinear(xi)
            self.face_xi.append(xi)
            self.face_phi.append(phi)
            self.face_dphi.append(dphi)
            self.face_N.append(Nf)
            self.face_dN.append(dNf)

    @property
    def n_dofs(self):
        return self.mesh.n_cells * self.n_dofs_cell

    # ------------------------------------------------------------------ geometry
    def cell_geometry(self, e):
        """points (P, 3), J (P, 3, 3), weights w det J (P,), J^-1 (P, 3, 3)."""
        Xv = self.mesh.cell_vertices(e)
        x = self.cell_N @ Xv
        J = np.einsum('pvl,vk->pkl', self.cell_dN, Xv)
        det = np.linalg.det(J)
        return x, J, self.cell_w * det, np.linalg.inv(J)

    def face_geometry(self, e, f):
        """points, J, outward unit normals (P, 3), surface weights (P,) on face f of cell e."""
        d, s = divmod(f, 2)
        t1, t2 = [a for a in range(3) if a != d]
        Xv = self.mesh.cell_vertices(e)
        x = self.face_N[f] @ Xv
        J = np.einsum('pvl,vk->pkl', self.face_dN[f], Xv)
        cr = np.cross(J[:, :, t1], J[:, :, t2])
        area = np.linalg.norm(cr, axis=1)
        orient = (2.0 * s - 1.0) * (-1.0 if d == 1 else 1.0)
        return x, J, orient * cr / area[:, None], self.face_w2 * area

    def _grad(self, dphi, J):
        """physical gradients (P, n3, 3) of the basis from reference ones and J (P, 3, 3)."""
        return np.einsum('pml,pim->pil', np.linalg.inv(J), dphi)

    def volume(self, e):
        return float(np.sum(self.cell_geometry(e)[2]))

    def face_area(self, e, f):
        return float(np.sum(self.face_geometry(e, f)[3]))

    def penalty_factor(self, e):
        lam = 0.0
        for f in range(6):
            w = 0.5 if self.mesh.boundary_type(e, f) == 'I' else 1.0
            lam += w * self.face_area(e, f)
        return lam / self.volume(e)

    def cell_points(self, e):
        return self.cell_geometry(e)[0]

    def face_points(self, e, f):
        return self.face_geometry(e, f)[0]

    def node_points(self, e):
        n = self.n
        iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing='ij')
        xi = np.stack([self.nodes[ix.ravel()], self.nodes[iy.ravel()], self.nodes[iz.ravel()]], axis=1)
        N, _ = _trilinear(xi)
        return N @ self.mesh.cell_vertices(e)

    def interpolate(self, func):
        C = self.mesh.n_cells
        out = np.zeros((C, self.ncomp, self.n ** 3))
        for e in range(C):
            v = np.asarray(func(self.node_points(e)), dtype=np.float64)
            out[e] = v.T if self.ncomp > 1 else v[None, :]
        return out.reshape(-1)

    # ------------------------------------------------------------- viscosity
    def viscosity_at_points(self, rheology, u=None, cells=None):
        C = self.mesh.n_cells
        nq3, nq2 = self.nq ** 3, self.nq ** 2
        nu_cell = np.zeros((C, nq3))
        nu_face = np.zeros((C, 6, nq2))
        needs_u = rheology['law'] == 'carreau'
        for e in (range(C) if cells is None else cells):
            ue = np.asarray(u).reshape(C, 3, self.n ** 3)[e] if needs_u else None
            x, J, W, _ = self.cell_geometry(e)
            grad = np.einsum('ci,pil->pcl', ue, self._grad(self.cell_dphi, J)) if needs_u else None
            nu_cell[e] = viscosity.evaluate(rheology, x, grad)
            if rheology['law'] == 'sinker' and rheology.get('projection', 'cell') == 'cell':
                nu_e = np.sum(W * nu_cell[e]) / np.sum(W)
                nu_cell[e] = nu_e
                nu_face[e] = nu_e
                continue
            for f in range(6):
                xf, Jf, _, _ = self.face_geometry(e, f)
                gf = np.einsum('ci,pil->pcl', ue, self._grad(self.face_dphi[f], Jf)) if needs_u else None
                nu_face[e, f] = viscosity.evaluate(rheology, xf, gf)
        return nu_cell, nu_face

    def _face_nubar(self, num, nup):
        if self.face_nu == 'max':
            return np.maximum(num, nup)
        if self.face_nu == 'arith':
            return 0.5 * (num + nup)
        return 2.0 * num * nup / (num + nup)

    def _tau(self, e, nb, num, nup):
        lam_m = self.penalty_factor(e)
        lam_p = lam_m if nb is None else self.penalty_factor(nb)
        return self.C_ip * (self.k + 1) ** 2 * max(lam_m, lam_p) * self._face_nubar(num, nup)

    # --------------------------------------------------------- element blocks
    def _vector_basis(self, phi, dphi_phys):
        P, n3 = phi.shape
        nc = self.ncomp
        V = np.zeros((P, nc * n3, nc))
        G = np.zeros((P, nc * n3, nc, 3))
        for c in range(nc):
            V[:, c * n3:(c + 1) * n3, c] = phi
            G[:, c * n3:(c + 1) * n3, c, :] = dphi_phys
        return V, G

    @staticmethod
    def _viscous_face(Vt, Gt, um, Gm, up, Gp, num, nup, tau, nvec, W):
        """Per-point normals nvec (P, 3); otherwise the flux of oracle.sipg."""
        avg = 0.5 * (um + up)
        a2 = 2.0 * num[:, None, None, None] * _sym(np.einsum('qbk,ql->qbkl', um - avg, nvec))
        T = 0.5 * (num[:, None, None, None] * Gm + nup[:, None, None, None] * Gp) \
            - tau[:, None, None, None] * np.einsum('qbk,ql->qbkl', um - up, nvec)
        flux = np.einsum('qbkl,ql->qbk', T + np.swapaxes(T, -1, -2), nvec)
        return -np.einsum('q,qakl,qbkl->ab', W, Gt, a2) - np.einsum('q,qak,qbk->ab', W, Vt, flux)

    @staticmethod
    def _poisson_face(qt, gt, pm, gm, pp, gp, tau, nvec, W):
        avg = 0.5 * (pm + pp)
        t2 = np.einsum('qb,ql->qbl', pm - avg, nvec)
        flux = np.einsum('qbl,ql->qb', 0.5 * (gm + gp), nvec) - tau[:, None] * (pm - pp)
        return -np.einsum('q,qal,qbl->ab', W, gt, t2) - np.einsum('q,qa,qb->ab', W, qt, flux)

    def blocks_of(self, e, nu_cell=None, nu_face=None, mass=0.0):
        mesh = self.mesh
        x, J, W, _ = self.cell_geometry(e)
        gphys = self._grad(self.cell_dphi, J)
        if self.ncomp == 3:
            V, G = self._vector_basis(self.cell_phi, gphys)
            own = np.einsum('q,qakl,qbkl->ab', W * 2.0 * nu_cell[e], G, _sym(G))
            if mass != 0.0:
                own += mass * np.einsum('q,qak,qbk->ab', W, V, V)
        else:
            own = np.einsum('q,qal,qbl->ab', W, gphys, gphys)
            if mass != 0.0:
                own += mass * np.einsum('q,qa,qb->ab', W, self.cell_phi, self.cell_phi)
        nbs = {}
        for f in range(6):
            d, s = divmod(f, 2)
            bt = mesh.boundary_type(e, f)
            if bt == 'N':
                continue
            _, Jf, nvec, Wf = self.face_geometry(e, f)
            gt = self._grad(self.face_dphi[f], Jf)
            if bt == 'I':
                nb = mesh.neighbor(e, f)
                fo = 2 * d + (1 - s)
                _, Jn, _, _ = self.face_geometry(nb, fo)
                gn = self._grad(self.face_dphi[fo], Jn)
            if self.ncomp == 3:
                Vt, Gt = self._vector_basis(self.face_phi[f], gt)
                num = nu_face[e, f]
                if bt == 'I':
                    nup = nu_face[nb, fo]
                    tau = self._tau(e, nb, num, nup)
                    Vn, Gn = self._vector_basis(self.face_phi[fo], gn)
                    zv, zg = np.zeros_like(Vt), np.zeros_like(Gt)
                    own += self._viscous_face(Vt, Gt, Vt, Gt, zv, zg, num, nup, tau, nvec, Wf)
                    nbs[f] = (nb, self._viscous_face(Vt, Gt, zv, zg, Vn, Gn, num, nup, tau, nvec, Wf))
                else:
                    tau = self._tau(e, None, num, num)
                    own += self._viscous_face(Vt, Gt, Vt, Gt, -Vt, Gt, num, num, tau, nvec, Wf)
            else:
                qt = self.face_phi[f]
                ones = np.ones(self.nq ** 2)
                if bt == 'I':
                    tau = self._tau(e, nb, ones, ones)
                    qn = self.face_phi[fo]
                    own += self._poisson_face(qt, gt, qt, gt, 0 * qt, 0 * gt, tau, nvec, Wf)
                    nbs[f] = (nb, self._poisson_face(qt, gt, 0 * qt, 0 * gt, qn, gn, tau, nvec, Wf))
                else:
                    tau = self._tau(e, None, ones, ones)
                    own += self._poisson_face(qt, gt, qt, gt, -qt, gt, tau, nvec, Wf)
        return own, nbs

    def rows(self, x, cells, nu_cell=None, nu_face=None, mass=0.0):
        """Rows of y = A x of the listed cells only (the viscosity of those cells and of
        their face neighbours must be set)."""
        m = self.n_dofs_cell
        X = np.asarray(x, dtype=np.float64).reshape(self.mesh.n_cells, m)
        out = []
        for e in cells:
            own, nbs = self.blocks_of(e, nu_cell, nu_face, mass)
            r = own @ X[e]
            for f, (nb, blk) in nbs.items():
                r = r + blk @ X[nb]
            out.append(r)
        return np.array(out)

    def apply(self, x, nu_cell=None, nu_face=None, mass=0.0):
        m = self.n_dofs_cell
        X = np.asarray(x, dtype=np.float64).reshape(self.mesh.n_cells, m)
        Y = np.zeros_like(X)
        for e in range(self.mesh.n_cells):
            own, nbs = self.blocks_of(e, nu_cell, nu_face, mass)
            Y[e] = own @ X[e]
            for f, (nb, blk) in nbs.items():
                Y[e] += blk @ X[nb]
        return Y.reshape(-1)

    def assemble(self, nu_cell=None, nu_face=None, mass=0.0):
        m = self.n_dofs_cell
        rows, cols, vals = [], [], []
        ii, jj = np.meshgrid(np.arange(m), np.arange(m), indexing='ij')
        for e in range(self.mesh.n_cells):
            own, nbs = self.blocks_of(e, nu_cell, nu_face, mass)
            rows.append(e * m + ii.ravel())
            cols.append(e * m + jj.ravel())
            vals.append(own.ravel())
            for f, (nb, blk) in nbs.items():
                rows.append(e * m + ii.ravel())
                cols.append(nb * m + jj.ravel())
                vals.append(blk.ravel())
        N = self.n_dofs
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(N, N)).tocsr()
