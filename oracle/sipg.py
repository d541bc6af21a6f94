"""Explicit SIPG operators on a box of affine hexahedra (oracle, test infrastructure).

What is computed
----------------
The element forms of Sec. 5, evaluated literally per element Omega_e, with the
exterior state u^+ taken from the neighbour (interior face) or from the mirror
principle (boundary face), then differentiated with respect to the nodal
coefficients to give explicit matrix blocks:

Viscous operator, Eq. (viscous_term_weak):
    v_h^e(v, u; nu) = (grad v, 2 nu eps(u))_e
                      - (grad v, 2 nu [(u - u^dag) (x) n]^S)_{de}
                      - (v, (tau_1^dag + tau_2^dag) . n)_{de}
  with the SIPG fluxes of Sec. 5.2:
    u^dag = {{u}},  tau_1^dag = {{nu grad u}} - tau [[u]],  tau_2^dag = (tau_1^dag)^T,
    [[u]] = u^- (x) n - u^+ (x) n.
  Optional mass term m (v, u)_e for the viscous-step operator (gamma_0/dt) M + A,
  Eq. (viscous_step_weak) with alpha_c = 0.

Pressure Poisson operator, Eq. (pressure_step_weak), left-hand side:
    (grad q, grad p)_e - (grad q, (p - {{p}}) n)_{de} - (q, ({{grad p}} - tau [[p]]) . n)_{de}
  READING: the paper prints "+ tau [[p]]", which summed over both sides of a
  face gives a negative (non-coercive) penalty; the viscous flux of Sec. 5.2
  carries "- tau [[u]]", and the standard SIPG sign is used here.

Boundary faces (mirror principle, Sec. 5.1, homogeneous data - the operator):
  Dirichlet: u^+ = -u^-, grad u^+ = grad u^-, nu^+ = nu^-;  Neumann: no term.

Penalty (READING, formula not printed; "according to Hillewaert 2013"):
  tau = C_IP (k+1)^2 max(Lambda^-, Lambda^+) nubar with Lambda_e from
  ``BoxMesh.penalty_factor``; nubar = max(nu^-, nu^+) pointwise (option 'max'),
  or the arithmetic / harmonic mean; the Poisson operator uses nubar = 1.

Sphere ("sinker") viscosity (READING): evaluated pointwise at the cell's Gauss
points, then projected element-locally in L2 onto a constant per cell (the
paper names element-local projection onto a discontinuous space as a viable
alternative to pointwise storage, Sec. 5.1) and stored at every cell and face
point of that cell. With the raw pointwise indicator the form is not coercive:
a face point inside a sphere next to cell points outside it makes the face
flux outweigh the cell term (a test keeps that finding). Option
``projection='pointwise'`` keeps the raw values.

Quadrature: k+1 Gauss-Legendre points per direction in cells and on faces; the
basis is Lagrange on k+1 Gauss-Lobatto nodes (Sec. 5). nu is stored at the
quadrature points (Eq. viscosity_pointwise): cell values nu_cell[e, q] with
q = (qz*n + qy)*n + qx, face values nu_face[e, f, q] of the cell's own side
with q = a + n*b over the face's tangential directions t1 < t2.

DoF layout: index ((e*ncomp + c)*n + iz)*n^2 + iy*n + ix.

Pins (tests/test_oracle_*.py): symmetry, rigid-body / constant null spaces,
positive definiteness, Galerkin consistency for a Q_2 field, brute-force
quadrature on one and two cells, and k+1 convergence.
"""
import numpy as np
import scipy.sparse as sp

from . import basis, quadrature, viscosity


def _sym(t):
    return 0.5 * (t + np.swapaxes(t, -1, -2))


class SIPG:
    """Explicit element blocks of the viscous (ncomp=3) or Poisson (ncomp=1) operator."""

    def __init__(self, mesh, k, ncomp, penalty_factor=1.0, face_nu='max', n_quad=None):
        if k < 1:
            raise ValueError("degree must be >= 1")
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
        # cell quadrature points, q = (qz*nq + qy)*nq + qx
        qz, qy, qx = np.meshgrid(np.arange(nq), np.arange(nq), np.arange(nq), indexing='ij')
        qx, qy, qz = qx.ravel(), qy.ravel(), qz.ravel()
        self.cell_xi = np.stack([self.gpts[qx], self.gpts[qy], self.gpts[qz]], axis=1)
        self.cell_w = self.gwts[qx] * self.gwts[qy] * self.gwts[qz]
        self.cell_phi, self.cell_dphi = basis.tensor_basis(self.nodes, self.cell_xi)
        # face quadrature points, q = a + nq*b along t1 < t2, for each of the 6 faces
        self.face_xi, self.face_phi, self.face_dphi = [], [], []
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
            self.face_xi.append(xi)
            self.face_phi.append(phi)
            self.face_dphi.append(dphi)

    # ------------------------------------------------------------------ geometry
    @property
    def n_dofs(self):
        return self.mesh.n_cells * self.n_dofs_cell

    def cell_points(self, e):
        return self.mesh.origin(e) + self.cell_xi * self.mesh.h

    def face_points(self, e, f):
        return self.mesh.origin(e) + self.face_xi[f] * self.mesh.h

    def node_points(self, e):
        n = self.n
        iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing='ij')
        xi = np.stack([self.nodes[ix.ravel()], self.nodes[iy.ravel()], self.nodes[iz.ravel()]], axis=1)
        return self.mesh.origin(e) + xi * self.mesh.h

    def all_node_points(self):
        return np.stack([self.node_points(e) for e in range(self.mesh.n_cells)])

    def _phys_grad(self, dphi):
        return dphi / self.mesh.h  # d/dx_l = (1/h_l) d/dxi_l for the affine box map

    # ----------------------------------------------------------- vector basis
    def _vector_basis(self, phi, dphi_phys):
        """V[p, a, k] and G[p, a, k, l] for a = c*n^3 + i, component c of phi_i e_c."""
        P, n3 = phi.shape
        nc = self.ncomp
        V = np.zeros((P, nc * n3, nc))
        G = np.zeros((P, nc * n3, nc, 3))
        for c in range(nc):
            V[:, c * n3:(c + 1) * n3, c] = phi
            G[:, c * n3:(c + 1) * n3, c, :] = dphi_phys
        return V, G

    # ------------------------------------------------------------- viscosity
    def viscosity_at_points(self, rheology, u=None, cells=None):
        """nu_cell (C, nq^3) and nu_face (C, 6, nq^2) per Eq. (viscosity_pointwise).

        For the Carreau-Yasuda law the gradient of the DoF vector u is taken on
        each side from that side's own cell (face values differ per side).
        ``cells`` restricts the evaluation to a subset (others stay zero)."""
        C = self.mesh.n_cells
        nq3, nq2 = self.nq ** 3, self.nq ** 2
        nu_cell = np.zeros((C, nq3))
        nu_face = np.zeros((C, 6, nq2))
        needs_u = rheology['law'] == 'carreau'
        if needs_u and u is None:
            raise ValueError("Carreau-Yasuda viscosity needs the velocity vector")
        for e in (range(C) if cells is None else cells):
            ue = None
            if needs_u:
                ue = np.asarray(u).reshape(C, 3, self.n ** 3)[e]
            grad = None
            if needs_u:
                dphi = self._phys_grad(self.cell_dphi)
                grad = np.einsum('ci,pil->pcl', ue, dphi)
            nu_cell[e] = viscosity.evaluate(rheology, self.cell_points(e), grad)
            if rheology['law'] == 'sinker' and rheology.get('projection', 'cell') == 'cell':
                # element-local L2 projection onto constants with the cell's Gauss rule
                nu_e = np.sum(self.cell_w * nu_cell[e]) / np.sum(self.cell_w)
                nu_cell[e] = nu_e
                nu_face[e] = nu_e
                continue
            for f in range(6):
                gf = None
                if needs_u:
                    gf = np.einsum('ci,pil->pcl', ue, self._phys_grad(self.face_dphi[f]))
                nu_face[e, f] = viscosity.evaluate(rheology, self.face_points(e, f), gf)
        return nu_cell, nu_face

    def _face_nubar(self, num, nup):
        if self.face_nu == 'max':
            return np.maximum(num, nup)
        if self.face_nu == 'arith':
            return 0.5 * (num + nup)
        if self.face_nu == 'harmonic':
            return 2.0 * num * nup / (num + nup)
        raise ValueError(f"unknown face viscosity mode {self.face_nu!r}")

    def _tau(self, e, nb, num, nup):
        """Penalty at the face points of cell e toward nb (None on the boundary)."""
        lam_m = self.mesh.penalty_factor(e)
        lam_p = lam_m if nb is None else self.mesh.penalty_factor(nb)
        return self.C_ip * (self.k + 1) ** 2 * max(lam_m, lam_p) * self._face_nubar(num, nup)

    # --------------------------------------------------------- element blocks
    def viscous_blocks(self, e, nu_cell, nu_face, mass=0.0):
        """Row blocks of cell e: (own block, {face f: (neighbour, block)})."""
        assert self.ncomp == 3
        mesh = self.mesh
        detJ = mesh.volume()
        W = self.cell_w * detJ
        V, G = self._vector_basis(self.cell_phi, self._phys_grad(self.cell_dphi))
        # cell term (grad v, 2 nu eps(u)) + mass (v, u)
        own = np.einsum('q,qakl,qbkl->ab', W * 2.0 * nu_cell[e], G, _sym(G))
        if mass != 0.0:
            own += mass * np.einsum('q,qak,qbk->ab', W, V, V)
        nbs = {}
        for f in range(6):
            d, s = divmod(f, 2)
            btype = mesh.boundary_type(e, f)
            if btype == 'N':
                continue  # homogeneous Neumann: the flux equals the (zero) data
            nvec = np.zeros(3)
            nvec[d] = 2.0 * s - 1.0
            Wf = self.face_w2 * mesh.face_area(d)
            Vt, Gt = self._vector_basis(self.face_phi[f], self._phys_grad(self.face_dphi[f]))
            num = nu_face[e, f]
            if btype == 'I':
                nb = mesh.neighbor(e, f)
                fo = 2 * d + (1 - s)  # the neighbour sees this face as its opposite face
                nup = nu_face[nb, fo]
                tau = self._tau(e, nb, num, nup)
                Vn, Gn = self._vector_basis(self.face_phi[fo], self._phys_grad(self.face_dphi[fo]))
                zero_v, zero_g = np.zeros_like(Vt), np.zeros_like(Gt)
                # own coefficients enter through u^-, the neighbour's through u^+
                own += self._viscous_face(Vt, Gt, Vt, Gt, zero_v, zero_g, num, nup, tau, nvec, Wf)
                nbs[f] = (nb, self._viscous_face(Vt, Gt, zero_v, zero_g, Vn, Gn, num, nup, tau, nvec, Wf))
            else:  # Dirichlet, mirror principle with homogeneous data
                tau = self._tau(e, None, num, num)
                own += self._viscous_face(Vt, Gt, Vt, Gt, -Vt, Gt, num, num, tau, nvec, Wf)
        return own, nbs

    @staticmethod
    def _viscous_face(Vt, Gt, um, Gm, up, Gp, num, nup, tau, nvec, W):
        """sum_q W_q [ -grad v : 2 nu^- sym((u^- - {{u}}) x n) - v . ((T + T^T) n) ],
        T = {{nu grad u}} - tau (u^- - u^+) x n, for trial states indexed by b."""
        avg = 0.5 * (um + up)
        a2 = 2.0 * num[:, None, None, None] * _sym(np.einsum('qbk,l->qbkl', um - avg, nvec))
        T = 0.5 * (num[:, None, None, None] * Gm + nup[:, None, None, None] * Gp) \
            - tau[:, None, None, None] * np.einsum('qbk,l->qbkl', um - up, nvec)
        flux = np.einsum('qbkl,l->qbk', T + np.swapaxes(T, -1, -2), nvec)
        return -np.einsum('q,qakl,qbkl->ab', W, Gt, a2) - np.einsum('q,qak,qbk->ab', W, Vt, flux)

    def poisson_blocks(self, e, mass=0.0):
        """Row blocks of cell e for the SIPG Laplacian (scalar, nu = 1)."""
        assert self.ncomp == 1
        mesh = self.mesh
        detJ = mesh.volume()
        W = self.cell_w * detJ
        phi = self.cell_phi
        g = self._phys_grad(self.cell_dphi)
        own = np.einsum('q,qal,qbl->ab', W, g, g)
        if mass != 0.0:
            own += mass * np.einsum('q,qa,qb->ab', W, phi, phi)
        nbs = {}
        ones = np.ones(self.nq ** 2)
        for f in range(6):
            d, s = divmod(f, 2)
            btype = mesh.boundary_type(e, f)
            if btype == 'N':
                continue
            nvec = np.zeros(3)
            nvec[d] = 2.0 * s - 1.0
            Wf = self.face_w2 * mesh.face_area(d)
            qt = self.face_phi[f]
            gt = self._phys_grad(self.face_dphi[f])
            if btype == 'I':
                nb = mesh.neighbor(e, f)
                fo = 2 * d + (1 - s)
                tau = self._tau(e, nb, ones, ones)
                qn = self.face_phi[fo]
                gn = self._phys_grad(self.face_dphi[fo])
                own += self._poisson_face(qt, gt, qt, gt, 0 * qt, 0 * gt, tau, nvec, Wf)
                nbs[f] = (nb, self._poisson_face(qt, gt, 0 * qt, 0 * gt, qn, gn, tau, nvec, Wf))
            else:
                tau = self._tau(e, None, ones, ones)
                own += self._poisson_face(qt, gt, qt, gt, -qt, gt, tau, nvec, Wf)
        return own, nbs

    @staticmethod
    def _poisson_face(qt, gt, pm, gm, pp, gp, tau, nvec, W):
        """sum_q W_q [ -grad q . (p^- - {{p}}) n - q ({{grad p}} - tau (p^- - p^+) n) . n ]."""
        avg = 0.5 * (pm + pp)
        t2 = np.einsum('qb,l->qbl', pm - avg, nvec)
        flux = np.einsum('qbl,l->qb', 0.5 * (gm + gp), nvec) - tau[:, None] * (pm - pp)
        return -np.einsum('q,qal,qbl->ab', W, gt, t2) - np.einsum('q,qa,qb->ab', W, qt, flux)

    # ------------------------------------------------------------ global ops
    def blocks(self, nu_cell=None, nu_face=None, mass=0.0, cells=None):
        cells = range(self.mesh.n_cells) if cells is None else cells
        out = {}
        for e in cells:
            if self.ncomp == 3:
                out[e] = self.viscous_blocks(e, nu_cell, nu_face, mass)
            else:
                out[e] = self.poisson_blocks(e, mass)
        return out

    def apply(self, x, nu_cell=None, nu_face=None, mass=0.0, cells=None):
        """y = A x element by element (rows of the listed cells only if given)."""
        m = self.n_dofs_cell
        X = np.asarray(x, dtype=np.float64).reshape(self.mesh.n_cells, m)
        cells = list(range(self.mesh.n_cells)) if cells is None else list(cells)
        Y = np.zeros((len(cells), m))
        for r, e in enumerate(cells):
            own, nbs = self.blocks(nu_cell, nu_face, mass, cells=[e])[e]
            Y[r] = own @ X[e]
            for f, (nb, blk) in nbs.items():
                Y[r] += blk @ X[nb]
        return Y.reshape(-1) if len(cells) == self.mesh.n_cells else Y

    def assemble(self, nu_cell=None, nu_face=None, mass=0.0):
        """Global sparse matrix (CSR) from the element row blocks."""
        m = self.n_dofs_cell
        rows, cols, vals = [], [], []
        ii, jj = np.meshgrid(np.arange(m), np.arange(m), indexing='ij')
        for e, (own, nbs) in self.blocks(nu_cell, nu_face, mass).items():
            rows.append(e * m + ii.ravel())
            cols.append(e * m + jj.ravel())
            vals.append(own.ravel())
            for f, (nb, blk) in nbs.items():
                rows.append(e * m + ii.ravel())
                cols.append(nb * m + jj.ravel())
                vals.append(blk.ravel())
        N = self.n_dofs
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, N))
        return A.tocsr()

    def interpolate(self, func):
        """Nodal interpolant of func(points (P,3)) -> (P, ncomp) at the GLL nodes."""
        C, n3 = self.mesh.n_cells, self.n ** 3
        pts = self.all_node_points().reshape(C * n3, 3)
        vals = np.asarray(func(pts)).reshape(C, n3, self.ncomp)
        return np.transpose(vals, (0, 2, 1)).reshape(-1)
