// Shared definitions of the libsipg CUDA sources (device side and host side).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

namespace sipg {

constexpr int kMaxN = 6;  // n = k + 1, degrees 1..5

// 1D tables of one degree, passed to kernels by value (lives in the
// kernel-parameter constant bank) and copied to shared memory on entry.
//  S[q*n + j]  = l_j(g_q): Lagrange basis on the n Gauss-Lobatto nodes at the
//                n Gauss-Legendre points (nodal values -> quadrature values)
//  Dg[q*n + p] = l'_p(g_q) for the Lagrange basis on the Gauss points
//                (collocation derivative at the quadrature points)
//  DS[q*n + j] = l'_j(g_q): derivative of the Gauss-Lobatto basis at Gauss points
//  dS0[j], dS1[j] = l'_j(0), l'_j(1): normal derivative at the cell faces
//  gw, gp       = Gauss weights / points on [0, 1];  gll = Gauss-Lobatto nodes
struct Tab {
  int n;
  double S[kMaxN * kMaxN];
  double Dg[kMaxN * kMaxN];
  double DS[kMaxN * kMaxN];
  double dS0[kMaxN], dS1[kMaxN];
  double gw[kMaxN], gp[kMaxN], gll[kMaxN];
  double M1[kMaxN * kMaxN];     // 1D mass matrix sum_q gw_q S[q][i] S[q][j] on [0, 1]
  double M1inv[kMaxN * kMaxN];  // its inverse
};

// 1D tables of the splitting-step forms of one velocity degree (n = k+1 Gauss
// points; the pressure basis has n-1 Gauss-Lobatto nodes), row-major [q][j]:
//  S, DS     velocity basis values / derivatives at the Gauss points
//  Dg        collocation derivative on the Gauss points
//  Sp, DSp   pressure basis values / derivatives at the velocity Gauss points
//  dS0, dS1  velocity basis derivatives at 0 and 1
//  lg0, lg1, dlg0, dlg1  Lagrange basis on the Gauss points: values and
//            derivatives at 0 and 1 (traces of fields given at Gauss points)
struct SplitTab {
  int n;
  double S[kMaxN * kMaxN], DS[kMaxN * kMaxN], Dg[kMaxN * kMaxN];
  double Sp[kMaxN * kMaxN], DSp[kMaxN * kMaxN];
  double dS0[kMaxN], dS1[kMaxN];
  double lg0[kMaxN], lg1[kMaxN], dlg0[kMaxN], dlg1[kMaxN];
  double gw[kMaxN], gp[kMaxN];  // Gauss weights and points on [0, 1]
  double Sinv[kMaxN * kMaxN];    // S^-1 [j][q]: the Lagrange basis on the Gauss points at the
                                 // Gauss-Lobatto nodes (Gauss-point values -> nodal values)
};

// Over-integration rule of the manufactured loads: nq Gauss points on [0, 1]
// (nq = n + 3) and the Gauss-Lobatto basis there, S[q*n + j] = l_j(gp_q).
constexpr int kMaxNQ = kMaxN + 3;
struct LoadTab {
  int n, nq;
  double S[kMaxN * kMaxNQ];
  double gw[kMaxNQ], gp[kMaxNQ];
};

// Global Gauss-Lobatto node grid of a continuous (cph) level on the box.
struct CgGrid {
  int nx, ny, nz, k, Gx, Gy, Gz, ncomp;
};
enum { CG_GATHER = 0, CG_SCATTER_SUM = 1, CG_PICK = 2, CG_PICK_T = 3 };

// Embedding matrices of the transfers (prolongation = interpolation of the
// coarse polynomial at the fine Gauss-Lobatto nodes), row-major [nf][nc].
struct TransferTab {
  int nf, nc;
  double E[kMaxN * kMaxN];      // p-transfer, or h-transfer child 0
  double E1[kMaxN * kMaxN];     // h-transfer child 1
};

// Geometry and discretisation of one level, passed by value to kernels.
// The cells are the active cells of an nx x ny x nz grid of equal boxes over
// [x0, x0 + extent]. The plain box (every cell active, no periodic direction)
// has no tables (nbr == nullptr): cell e is grid cell e and neighbours follow
// from the grid indices. Otherwise (cells removed, e.g. the channel behind a
// backward-facing step, or periodic directions) three device tables describe
// the topology:
//   nbr[e*6 + f]  >= 0: the cell across face f (periodic directions wrap);
//                 <  0: a boundary face, v = -1 - nbr with boundary id v & 7
//                       (0..5 the grid's sides -x,+x,-y,+y,-z,+z, 6 a face
//                       against a removed cell) and boundary-face number v >> 3
//   cgrid[e]      grid index (ix + nx (iy + ny iz)) of active cell e
//   gcell[i]      active index of grid cell i, or -1 for a removed cell
//   bface[b]      e*6 + f of boundary face b
// Boundary faces of the plain box are numbered side by side (-x first), each
// side lexicographic over its tangential cell indices t1 < t2.
struct LevelGeom {
  int nx, ny, nz;
  int ncells;
  double h[3];
  double ih[3];     // 1 / h, precomputed on the host (no FP64 division on the device)
  int bc[7];        // 0 = Dirichlet, 1 = Neumann, per boundary id
  double cip;       // penalty factor C_IP
  int face_nu;      // 0 max, 1 arithmetic, 2 harmonic
  double x0[3];     // lower corner of the grid
  int nbf;          // boundary faces
  const int* nbr;   // topology tables (nullptr: the plain box)
  const int* cgrid;
  const int* gcell;
  const int* bface;
};

__host__ __device__ inline void cell_ijk(const LevelGeom& g, int e, int* ijk) {
  const int i = g.cgrid ? g.cgrid[e] : e;
  ijk[0] = i % g.nx;
  ijk[1] = (i / g.nx) % g.ny;
  ijk[2] = i / (g.nx * g.ny);
}

// active index of grid cell (i, j, k) (in range), -1 if removed
__host__ __device__ inline int grid_cell(const LevelGeom& g, int i, int j, int k) {
  const int gi = (k * g.ny + j) * g.nx + i;
  return g.gcell ? g.gcell[gi] : gi;
}

__host__ __device__ inline int cell_neighbor(const LevelGeom& g, int e, int f) {
  if (g.nbr) {
    const int v = g.nbr[e * 6 + f];
    return v >= 0 ? v : -1;
  }
  const int d = f >> 1, s = f & 1;
  int ijk[3] = {e % g.nx, (e / g.nx) % g.ny, e / (g.nx * g.ny)};
  const int dims[3] = {g.nx, g.ny, g.nz};
  ijk[d] += s ? 1 : -1;
  if (ijk[d] < 0 || ijk[d] >= dims[d]) return -1;
  return (ijk[2] * g.ny + ijk[1]) * g.nx + ijk[0];
}

// Compile-time variants for kernels instantiated per kind of grid (TOPO: the
// topology tables are present); the plain box keeps its arithmetic path.
template <bool TOPO>
__host__ __device__ inline int cell_neighbor_t(const LevelGeom& g, int e, int f) {
  if (TOPO) {
    const int v = g.nbr[e * 6 + f];
    return v >= 0 ? v : -1;
  }
  const int d = f >> 1, s = f & 1;
  int ijk[3] = {e % g.nx, (e / g.nx) % g.ny, e / (g.nx * g.ny)};
  const int dims[3] = {g.nx, g.ny, g.nz};
  ijk[d] += s ? 1 : -1;
  if (ijk[d] < 0 || ijk[d] >= dims[d]) return -1;
  return (ijk[2] * g.ny + ijk[1]) * g.nx + ijk[0];
}
template <bool TOPO>
__host__ __device__ inline int face_bc_t(const LevelGeom& g, int e, int f) {
  return TOPO ? g.bc[(-1 - g.nbr[e * 6 + f]) & 7] : g.bc[f];
}

// boundary id of the boundary face (e, f) (the grid side f on the plain box)
__host__ __device__ inline int boundary_id(const LevelGeom& g, int e, int f) {
  return g.nbr ? ((-1 - g.nbr[e * 6 + f]) & 7) : f;
}

// boundary condition (0 Dirichlet, 1 Neumann) of the boundary face (e, f)
__host__ __device__ inline int face_bc(const LevelGeom& g, int e, int f) { return g.bc[boundary_id(g, e, f)]; }

// Wall velocity handed to the form launchers: `side`, 18 HOST doubles (a constant
// vector per grid side -x,+x,-y,+y,-z,+z; faces against removed cells take zero)
// or NULL (zero), and optionally `pts`, DEVICE values at the Gauss points of every
// boundary face ([nbf][n^2][3], see LevelGeom), which take precedence.
struct WallArg {
  const double* side;
  const double* pts;
  WallArg(const double* s = nullptr, const double* p = nullptr) : side(s), pts(p) {}
};

// Penalty geometry factor Lambda_e = sum_f w_f |f| / |Omega_e| with w_f = 1/2
// on interior and 1 on boundary faces (box cells: |f| / |Omega_e| = 1 / h_d).
__host__ __device__ inline double penalty_lambda(const LevelGeom& g, int e) {
  double lam = 0.0;
  for (int f = 0; f < 6; ++f) {
    const double w = cell_neighbor(g, e, f) >= 0 ? 0.5 : 1.0;
    lam += w * g.ih[f >> 1];
  }
  return lam;
}

template <bool TOPO>
__host__ __device__ inline double penalty_lambda_t(const LevelGeom& g, int e) {
  double lam = 0.0;
  for (int f = 0; f < 6; ++f) {
    const double w = cell_neighbor_t<TOPO>(g, e, f) >= 0 ? 0.5 : 1.0;
    lam += w * g.ih[f >> 1];
  }
  return lam;
}

}  // namespace sipg
