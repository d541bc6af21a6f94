"""Structured grids of affine hexahedra (oracle, test infrastructure).

Sec. 5: the domain is split into N_e non-overlapping hexahedra. Here the cells
are the active cells of a grid of nx*ny*nz equal boxes over [lo, lo + extent]
(the plain box: every cell active, lo = 0). Each cell maps from the reference
cube [0,1]^3 by x = origin + h * xi (affine, diagonal Jacobian). Active cells
are numbered in grid order, x fastest: on the plain box e = (ez*ny + ey)*nx + ex.

Removed cells describe domains such as the channel behind a backward-facing
step (Sec. 7: the grid over the channel's bounding box without the solid block
below the inlet); a periodic direction joins the first and last cell layers as
face neighbours.

Faces of a cell are numbered f = 2*d + s: d the normal direction, s = 0 the
face at xi_d = 0 (outward normal -e_d), s = 1 the face at xi_d = 1 (normal
+e_d). A boundary face carries a boundary id: 0..5 when it lies on the grid's
side -x, +x, -y, +y, -z, +z, 6 when it faces a removed cell. Each id has a type
'D' (Dirichlet) or 'N' (Neumann): bc lists six (plain box) or seven entries.

The penalty geometry factor follows the reading of Sec. 5.1/5.2 ("tau after
Hillewaert 2013", formula not printed): Lambda_e = sum_f w_f |f| / |Omega_e|
with w_f = 1/2 on interior faces and 1 on boundary faces.
"""
import numpy as np


class BoxMesh:
    def __init__(self, nx, ny, nz, extent=(1.0, 1.0, 1.0), bc=('D',) * 6, lo=(0.0, 0.0, 0.0), active=None,
                 periodic=(False, False, False)):
        self.n_cells_dir = (int(nx), int(ny), int(nz))
        self.extent = tuple(float(v) for v in extent)
        self.lo = np.array([float(v) for v in lo])
        self.h = np.array([self.extent[d] / self.n_cells_dir[d] for d in range(3)])
        bc = tuple(bc)
        if len(bc) == 6:
            bc = bc + ('D',)
        if len(bc) != 7 or any(b not in ('D', 'N') for b in bc):
            raise ValueError("bc must list six or seven entries from {'D', 'N'}")
        self.bc = bc
        self.periodic = tuple(bool(p) for p in periodic)
        for d in range(3):
            if self.periodic[d] and self.n_cells_dir[d] < 2:
                raise ValueError("a periodic direction needs two cells or more")
        G = int(np.prod(self.n_cells_dir))
        if active is None:
            self.active = np.ones(G, dtype=bool)
        else:
            self.active = np.asarray(active, dtype=bool).reshape(-1).copy()
            if self.active.size != G:
                raise ValueError("active: (nz, ny, nx) flags expected")
        self.grid_of = np.nonzero(self.active)[0]                 # active cell -> grid index
        self.cell_of = np.full(G, -1, dtype=np.int64)             # grid index -> active cell
        self.cell_of[self.grid_of] = np.arange(self.grid_of.size)
        if self.grid_of.size == 0:
            raise ValueError("no active cell")

    @property
    def n_cells(self):
        return int(self.grid_of.size)

    @property
    def plain(self):
        """Every cell active and no periodic direction."""
        return bool(self.active.all()) and not any(self.periodic)

    def cell_ijk(self, e):
        nx, ny, _ = self.n_cells_dir
        g = int(self.grid_of[e])
        return (g % nx, (g // nx) % ny, g // (nx * ny))

    def cell_index(self, ijk):
        """Active cell at grid position ijk, or None for a removed cell."""
        nx, ny, _ = self.n_cells_dir
        c = int(self.cell_of[(ijk[2] * ny + ijk[1]) * nx + ijk[0]])
        return c if c >= 0 else None

    def origin(self, e):
        return self.lo + np.array(self.cell_ijk(e), dtype=np.float64) * self.h

    def volume(self):
        return float(np.prod(self.h))

    def face_area(self, d):
        t = [a for a in range(3) if a != d]
        return float(self.h[t[0]] * self.h[t[1]])

    def _across(self, e, f):
        """(grid position across face f, boundary id or None)."""
        d, s = divmod(f, 2)
        ijk = list(self.cell_ijk(e))
        ijk[d] += 1 if s == 1 else -1
        if ijk[d] < 0 or ijk[d] >= self.n_cells_dir[d]:
            if not self.periodic[d]:
                return None, f
            ijk[d] %= self.n_cells_dir[d]
        if self.cell_index(ijk) is None:
            return None, 6
        return ijk, None

    def neighbor(self, e, f):
        """Cell across face f of cell e, or None on the boundary."""
        ijk, _ = self._across(e, f)
        return None if ijk is None else self.cell_index(ijk)

    def boundary_id(self, e, f):
        """Boundary id of face f of cell e (None for an interior face)."""
        return self._across(e, f)[1]

    def boundary_type(self, e, f):
        """'I' for an interior face, else the type of its boundary id."""
        b = self.boundary_id(e, f)
        return 'I' if b is None else self.bc[b]

    def boundary_faces(self):
        """[(e, f)] of every boundary face, in cell order, faces -x..+z within a cell."""
        return [(e, f) for e in range(self.n_cells) for f in range(6) if self.boundary_id(e, f) is not None]

    def penalty_factor(self, e):
        area = 0.0
        for f in range(6):
            w = 0.5 if self.neighbor(e, f) is not None else 1.0
            area += w * self.face_area(f // 2)
        return area / self.volume()

    def with_bc(self, bc):
        """The same cells with other boundary types."""
        return BoxMesh(*self.n_cells_dir, extent=self.extent, bc=bc, lo=self.lo, active=self.active,
                       periodic=self.periodic)

    def coarsen(self):
        nx, ny, nz = self.n_cells_dir
        if nx % 2 or ny % 2 or nz % 2:
            raise ValueError("cannot coarsen an odd number of cells")
        if any(p and n // 2 < 2 for p, n in zip(self.periodic, self.n_cells_dir)):
            raise ValueError("a periodic direction would keep fewer than two cells")
        A = self.active.reshape(nz, ny, nx)
        blocks = A.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).sum(axis=(1, 3, 5))
        if np.any((blocks > 0) & (blocks < 8)):
            raise ValueError("a 2x2x2 block mixes active and removed cells")
        return BoxMesh(nx // 2, ny // 2, nz // 2, self.extent, self.bc, lo=self.lo, active=blocks == 8,
                       periodic=self.periodic)
