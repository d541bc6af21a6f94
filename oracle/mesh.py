"""Structured box of affine hexahedra (oracle, test infrastructure).

Sec. 5: the domain is split into N_e non-overlapping hexahedra. Here the domain
is the box [0,Lx] x [0,Ly] x [0,Lz] cut into nx*ny*nz equal cells, numbered
lexicographically with x fastest: e = (ez*ny + ey)*nx + ex. Each cell maps from
the reference cube [0,1]^3 by x = origin + h * xi (affine, diagonal Jacobian).

Faces of a cell are numbered f = 2*d + s: d the normal direction, s = 0 the
face at xi_d = 0 (outward normal -e_d), s = 1 the face at xi_d = 1 (normal
+e_d). Box faces carry a boundary type: 'D' (Dirichlet) or 'N' (Neumann),
listed in the same order (-x, +x, -y, +y, -z, +z).

The penalty geometry factor follows the reading of Sec. 5.1/5.2 ("tau after
Hillewaert 2013", formula not printed): Lambda_e = sum_f w_f |f| / |Omega_e|
with w_f = 1/2 on interior faces and 1 on boundary faces.
"""
import numpy as np


class BoxMesh:
    def __init__(self, nx, ny, nz, extent=(1.0, 1.0, 1.0), bc=('D',) * 6):
        self.n_cells_dir = (int(nx), int(ny), int(nz))
        self.extent = tuple(float(v) for v in extent)
        self.h = np.array([self.extent[d] / self.n_cells_dir[d] for d in range(3)])
        if len(bc) != 6 or any(b not in ('D', 'N') for b in bc):
            raise ValueError("bc must list six entries from {'D', 'N'}")
        self.bc = tuple(bc)

    @property
    def n_cells(self):
        nx, ny, nz = self.n_cells_dir
        return nx * ny * nz

    def cell_ijk(self, e):
        nx, ny, _ = self.n_cells_dir
        return (e % nx, (e // nx) % ny, e // (nx * ny))

    def cell_index(self, ijk):
        nx, ny, _ = self.n_cells_dir
        return (ijk[2] * ny + ijk[1]) * nx + ijk[0]

    def origin(self, e):
        return np.array(self.cell_ijk(e), dtype=np.float64) * self.h

    def volume(self):
        return float(np.prod(self.h))

    def face_area(self, d):
        t = [a for a in range(3) if a != d]
        return float(self.h[t[0]] * self.h[t[1]])

    def neighbor(self, e, f):
        """Cell across face f of cell e, or None on the boundary."""
        d, s = divmod(f, 2)
        ijk = list(self.cell_ijk(e))
        ijk[d] += 1 if s == 1 else -1
        if ijk[d] < 0 or ijk[d] >= self.n_cells_dir[d]:
            return None
        return self.cell_index(ijk)

    def boundary_type(self, e, f):
        """'I' for an interior face, else the box face's type."""
        return 'I' if self.neighbor(e, f) is not None else self.bc[f]

    def penalty_factor(self, e):
        area = 0.0
        for f in range(6):
            w = 0.5 if self.neighbor(e, f) is not None else 1.0
            area += w * self.face_area(f // 2)
        return area / self.volume()

    def coarsen(self):
        nx, ny, nz = self.n_cells_dir
        if nx % 2 or ny % 2 or nz % 2:
            raise ValueError("cannot coarsen an odd number of cells")
        return BoxMesh(nx // 2, ny // 2, nz // 2, self.extent, self.bc)
