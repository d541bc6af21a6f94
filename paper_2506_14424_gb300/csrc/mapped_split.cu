// Forms of one step of the projection scheme on trilinear (non-affine)
// hexahedra - the jittered backward-facing-step channel - Sec. 3.2 / 5.1,
// Alg. 1 on the general hexahedra of Sec. 5. Same forms as split.cu, with the
// geometry of each quadrature point evaluated from the cell's 8 vertices
// (mapped_geom.cuh): W = w det J, grad = J^-T grad_xi, per-point outward unit
// normals and surface weights on the faces:
//   mconv_kernel     C_a = c_h(phi_a, u; u), Eq. (convective_term_weak)
//   mppe_bnd_kernel  h_p - (gamma0/dt) g_uhat.n at the Gauss points of every wall
//                    face, Eqs. (pressure_Neumann_BC), (guhat_consistent_BC)
//   mppe_rhs_kernel  (gamma0/dt)[(grad q, uhat) - (q, {{uhat}}.n)], Eq. (pressure_step_weak)
//   mproj_rhs_kernel (div v, p) - (v, {{p}} n), Eq. (projection_step_weak)
//   mvisc_dir_kernel Dirichlet wall-data terms of the SIPG viscous form
//   mcfl_kernel      max over Gauss points of |J^-1 u|, Eq. (CFL_timestep_selection)
//   mmass_kernel     coeff M x and (coeff M)^-1 x: with as many Gauss points as
//                    nodes the interpolation S to the Gauss points is square and
//                    invertible, so M = S^T diag(w det J) S and
//                    M^-1 = S^-1 diag(1 / (w det J)) S^-T exactly (tensor-product
//                    sweeps with S1^-1 per direction), for any cell shape
//   mbpoints_kernel  positions of the Gauss points of every boundary face
// FP64, one CTA per cell (per wall face for mppe_bnd), one thread per tensor
// entry of each sweep; each CTA writes only its own rows.
// The element-local L2 projection onto Q_k of Gauss-point values (vorticity,
// viscosity in the pressure datum) is the polynomial through those values on
// trilinear cells too: (S^T W S)^-1 S^T W f = S^-1 f.
#include "kernels.cuh"
#include "mapped_geom.cuh"
#include "sweeps.cuh"

#include <algorithm>

namespace sipg {
namespace {

using namespace sweeps;
using namespace mgeo;

// J^-1 and the weight w det J at cell Gauss point q
__device__ __forceinline__ double cell_geom(const double (*X)[3], const SplitTab& tab, int q, int n, double Ji[3][3]) {
  const int qx = q % n, qy = (q / n) % n, qz = q / (n * n);
  double J[3][3];
  trilinear_jac(X, tab.gp[qx], tab.gp[qy], tab.gp[qz], J);
  const double det = inverse3(J, Ji);
  return tab.gw[qx] * tab.gw[qy] * tab.gw[qz] * det;
}

// J^-1, the outward unit normal and the surface weight at Gauss point p of face (d, s)
__device__ __forceinline__ double face_geom(const double (*X)[3], const SplitTab& tab, int d, int s, int p, int n,
                                            double Ji[3][3], double nrm[3], double* pos = nullptr) {
  int t1, t2;
  face_dirs(d, &t1, &t2);
  double xi[3];
  xi[d] = s ? 1.0 : 0.0;
  xi[t1] = tab.gp[p % n];
  xi[t2] = tab.gp[p / n];
  double J[3][3];
  trilinear_jac(X, xi[0], xi[1], xi[2], J, pos);
  inverse3(J, Ji);
  const double ta[3] = {J[0][t1], J[1][t1], J[2][t1]}, tb[3] = {J[0][t2], J[1][t2], J[2][t2]};
  const double c[3] = {ta[1] * tb[2] - ta[2] * tb[1], ta[2] * tb[0] - ta[0] * tb[2], ta[0] * tb[1] - ta[1] * tb[0]};
  const double area = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
  const double orient = (2.0 * s - 1.0) * (d == 1 ? -1.0 : 1.0);
  for (int k = 0; k < 3; ++k) nrm[k] = c[k] * orient / area;
  return tab.gw[p % n] * tab.gw[p / n] * area;
}

// physical gradient sum_m r_m J^-1[m][l]
__device__ __forceinline__ void to_phys(const double r[3], const double Ji[3][3], double out[3]) {
  for (int l = 0; l < 3; ++l) out[l] = r[0] * Ji[0][l] + r[1] * Ji[1][l] + r[2] * Ji[2][l];
}

// values of the layer nodes of a nodal field at the face Gauss points (2D S sweeps)
template <int N>
__device__ __forceinline__ void face_values(const double* __restrict__ U, int d, int s, const STabSm& T, double* out,
                                            double* tmp) {
  constexpr int N2 = N * N;
  for (int p = threadIdx.x; p < N2; p += blockDim.x) out[p] = U[fnode(d, s, p % N, p / N, N)];
  __syncthreads();
  sweep<N, N, 1, 0, N, false>(T.S, N, out, tmp);
  __syncthreads();
  sweep<N, N, 1, 1, N, false>(T.S, N, tmp, out);
  __syncthreads();
}

// add the transposed face values of coefficients cf (Gauss points) to the layer nodes of Y
template <int N>
__device__ __forceinline__ void face_values_t(const double* cf, int d, int s, const STabSm& T, double* Y, double* tmp,
                                              double* tmp2) {
  constexpr int N2 = N * N;
  sweep<N, N, 1, 0, N, true>(T.S, N, cf, tmp);
  __syncthreads();
  sweep<N, N, 1, 1, N, true>(T.S, N, tmp, tmp2);
  __syncthreads();
  for (int p = threadIdx.x; p < N2; p += blockDim.x) Y[fnode(d, s, p % N, p / N, N)] += tmp2[p];
  __syncthreads();
}

// --------------------------------------------------------------- convective
template <int N>
__global__ void __launch_bounds__(kSplitThreads) mconv_kernel(LevelGeom g, SplitTab tab, Wall wall,
                                                              const double* __restrict__ verts,
                                                              const double* __restrict__ u, double* __restrict__ y) {
  constexpr int N3 = N * N * N, N2 = N * N;
  __shared__ STabSm T;
  __shared__ double X[8][3];
  __shared__ double U[3][N3], Q[3][N3], G[3][3][N3], CV[3][N3], T0[N3], T1[N3], OUT[3][N3];
  __shared__ double UM[3][N2], UP[3][N2], FT[N2], FL[3][N2], FR[N2];
  const int e = blockIdx.x;
  load_tab(tab, T);
  load_cell_vertices(g, verts, e, X);
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) U[i / N3][i % N3] = u[(size_t)e * 3 * N3 + i];
  __syncthreads();
  for (int c = 0; c < 3; ++c) sweep3<N, N, false>(T.S, N, U[c], T0, T1, Q[c]);
  for (int c = 0; c < 3; ++c)
    for (int m = 0; m < 3; ++m) sweep_dir<N, false>(m, T.Dg, Q[c], G[c][m]);
  __syncthreads();
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    double Ji[3][3];
    const double W = cell_geom(X, tab, q, N, Ji);
    for (int c = 0; c < 3; ++c) {
      const double r[3] = {G[c][0][q], G[c][1][q], G[c][2][q]};
      double gp[3];
      to_phys(r, Ji, gp);
      CV[c][q] = W * (Q[0][q] * gp[0] + Q[1][q] * gp[1] + Q[2][q] * gp[2]);
    }
  }
  __syncthreads();
  for (int c = 0; c < 3; ++c) sweep3<N, N, true>(T.S, N, CV[c], T0, T1, OUT[c]);
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    const int nb = cell_neighbor(g, e, f);
    for (int c = 0; c < 3; ++c) {
      face_values<N>(U[c], d, s, T, UM[c], FT);
      if (nb >= 0) face_values<N>(u + (size_t)nb * 3 * N3 + c * N3, d, 1 - s, T, UP[c], FT);
    }
    const bool dir = nb < 0 && face_bc(g, e, f) == 0;
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      double Ji[3][3], nrm[3];
      const double Wf = face_geom(X, tab, d, s, p, N, Ji, nrm);
      double um[3], up[3];
      for (int c = 0; c < 3; ++c) {
        um[c] = UM[c][p];
        up[c] = nb >= 0 ? UP[c][p] : (dir ? -um[c] + 2.0 * wall_val(wall, g, e, f, p, c, N2) : um[c]);
      }
      const double wn = 0.5 * ((um[0] + up[0]) * nrm[0] + (um[1] + up[1]) * nrm[1] + (um[2] + up[2]) * nrm[2]);
      const double sg = wn > 0.0 ? 1.0 : (wn < 0.0 ? -1.0 : 0.0);
      for (int c = 0; c < 3; ++c) FL[c][p] = Wf * wn * 0.5 * (1.0 - sg) * (up[c] - um[c]);
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) face_values_t<N>(FL[c], d, s, T, OUT[c], FT, FR);
  }
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) y[(size_t)e * 3 * N3 + i] = OUT[i / N3][i % N3];
}

// ----------------------------------------------------- PPE wall datum
struct MPpeBnd {
  PpeBndArgs a;
  RheologyDev rh;  // constant or Carreau-Yasuda
};

__device__ __forceinline__ double eta_law(const RheologyDev& r, const double G[3][3]) {
  if (r.law == 0) return r.nu;
  double ee = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      const double v = 0.5 * (G[k][l] + G[l][k]);
      ee += v * v;
    }
  const double gdot = sqrt(2.0 * ee);
  return r.eta_inf + (r.eta0 - r.eta_inf) * pow(r.kappa + pow(r.lambda * gdot, r.a), (r.b - 1.0) / r.a);
}

// value, d/dxi_d, d/dxi_t1, d/dxi_t2 at the face Gauss points of a field given at
// the cell Gauss points (its Q_k interpolant): out[0..3] (N^2 each)
template <int N>
__device__ __forceinline__ void gauss_face_eval(const double* F, int d, int s, const STabSm& T, double* out) {
  constexpr int N2 = N * N;
  trace<N>(F, T.lg[s], d, out);
  trace<N>(F, T.dlg[s], d, out + N2);
  __syncthreads();
  sweep<N, N, 1, 0, N, false>(T.Dg, N, out, out + 2 * N2);
  sweep<N, N, 1, 1, N, false>(T.Dg, N, out, out + 3 * N2);
  __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(kSplitThreads) mppe_bnd_kernel(LevelGeom g, SplitTab tab, Wall wall, MPpeBnd pb,
                                                                 const double* __restrict__ verts,
                                                                 const double* __restrict__ u0,
                                                                 const double* __restrict__ u1,
                                                                 double* __restrict__ sb) {
  constexpr int N3 = N * N * N, N2 = N * N;
  __shared__ STabSm T;
  __shared__ double X[8][3];
  __shared__ double U[3][N3], Q[3][N3], G[3][3][N3], T0[N3], T1[N3], W3[3][N3];
  __shared__ double TR[3][N2], TG[3][3][N2], FE[4][4 * N2], ACC[N2];
  int e, f;
  bface_cell(g, blockIdx.x, &e, &f);
  if (face_bc(g, e, f) != 0) {  // velocity Neumann (pressure Dirichlet): no datum
    for (int p = threadIdx.x; p < N2; p += blockDim.x) sb[(size_t)blockIdx.x * N2 + p] = 0.0;
    return;
  }
  const int d = f >> 1, s = f & 1;
  load_tab(tab, T);
  load_cell_vertices(g, verts, e, X);
  __syncthreads();
  for (int p = threadIdx.x; p < N2; p += blockDim.x) {
    double Ji[3][3], nrm[3];
    face_geom(X, tab, d, s, p, N, Ji, nrm);
    double gn = 0.0;
    for (int c = 0; c < 3; ++c) gn += wall_val(wall, g, e, f, p, c, N2) * nrm[c];
    ACC[p] = pb.a.gn_coef * gn;
  }
  __syncthreads();
  // convective terms n.(u.grad)u of each history, weight beta_i - betabar_i
  for (int h = 0; h < pb.a.n_hist; ++h) {
    const double* uh = h == 0 ? u0 : u1;
    if (pb.a.wconv[h] == 0.0) continue;
    for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) U[i / N3][i % N3] = uh[(size_t)e * 3 * N3 + i];
    __syncthreads();
    for (int c = 0; c < 3; ++c) sweep3<N, N, false>(T.S, N, U[c], T0, T1, Q[c]);
    for (int c = 0; c < 3; ++c)
      for (int m = 0; m < 3; ++m) sweep_dir<N, false>(m, T.Dg, Q[c], G[c][m]);
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
      trace<N>(Q[c], T.lg[s], d, TR[c]);
      for (int m = 0; m < 3; ++m) trace<N>(G[c][m], T.lg[s], d, TG[c][m]);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      double Ji[3][3], nrm[3];
      face_geom(X, tab, d, s, p, N, Ji, nrm);
      double cv = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double r[3] = {TG[c][0][p], TG[c][1][p], TG[c][2][p]};
        double gp[3];
        to_phys(r, Ji, gp);
        cv += nrm[c] * (TR[0][p] * gp[0] + TR[1][p] * gp[1] + TR[2][p] * gp[2]);
      }
      ACC[p] += pb.a.wconv[h] * cv;
    }
    __syncthreads();
  }
  if (pb.a.visc) {
    // u^dd = sum_i betabar_i u^{n-i}
    for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) {
      const size_t k = (size_t)e * 3 * N3 + i;
      double v = pb.a.betabar[0] * u0[k];
      if (pb.a.betabar[1] != 0.0) v += pb.a.betabar[1] * u1[k];
      U[i / N3][i % N3] = v;
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) sweep3<N, N, false>(T.S, N, U[c], T0, T1, Q[c]);
    for (int c = 0; c < 3; ++c)
      for (int m = 0; m < 3; ++m) sweep_dir<N, false>(m, T.Dg, Q[c], G[c][m]);
    __syncthreads();
    // vorticity and viscosity at the Gauss points (their L2 projections onto Q_k)
    for (int q = threadIdx.x; q < N3; q += blockDim.x) {
      double Ji[3][3];
      cell_geom(X, tab, q, N, Ji);
      double Gq[3][3];
      for (int c = 0; c < 3; ++c) {
        const double r[3] = {G[c][0][q], G[c][1][q], G[c][2][q]};
        to_phys(r, Ji, Gq[c]);
      }
      W3[0][q] = Gq[2][1] - Gq[1][2];
      W3[1][q] = Gq[0][2] - Gq[2][0];
      W3[2][q] = Gq[1][0] - Gq[0][1];
      T0[q] = eta_law(pb.rh, Gq);
    }
    __syncthreads();
    for (int j = 0; j < 3; ++j) gauss_face_eval<N>(W3[j], d, s, T, FE[j]);
    gauss_face_eval<N>(T0, d, s, T, FE[3]);
    for (int c = 0; c < 3; ++c)
      for (int m = 0; m < 3; ++m) trace<N>(G[c][m], T.lg[s], d, TG[c][m]);
    __syncthreads();
    int t1, t2;
    face_dirs(d, &t1, &t2);
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      double Ji[3][3], nrm[3];
      face_geom(X, tab, d, s, p, N, Ji, nrm);
      double gw[4][3];  // physical gradients of omega_0..2 and nu
      for (int j = 0; j < 4; ++j) {
        double r[3];
        r[d] = FE[j][N2 + p];
        r[t1] = FE[j][2 * N2 + p];
        r[t2] = FE[j][3 * N2 + p];
        to_phys(r, Ji, gw[j]);
      }
      const double curl[3] = {gw[2][1] - gw[1][2], gw[0][2] - gw[2][0], gw[1][0] - gw[0][1]};
      double Gf[3][3];
      for (int c = 0; c < 3; ++c) {
        const double r[3] = {TG[c][0][p], TG[c][1][p], TG[c][2][p]};
        to_phys(r, Ji, Gf[c]);
      }
      const double nu = eta_law(pb.rh, Gf);
      double ncurl = 0.0, epsgrad = 0.0;
      for (int k = 0; k < 3; ++k) {
        ncurl += nrm[k] * curl[k];
        for (int l = 0; l < 3; ++l) epsgrad += nrm[k] * 0.5 * (Gf[k][l] + Gf[l][k]) * gw[3][l];
      }
      ACC[p] += -nu * ncurl + 2.0 * epsgrad;
    }
    __syncthreads();
  }
  for (int p = threadIdx.x; p < N2; p += blockDim.x) sb[(size_t)blockIdx.x * N2 + p] = ACC[p];
}

// ------------------------------------------------------ PPE right-hand side
template <int N>
__global__ void __launch_bounds__(kSplitThreads) mppe_rhs_kernel(LevelGeom g, SplitTab tab, double coef,
                                                                 const double* __restrict__ verts,
                                                                 const double* __restrict__ uh,
                                                                 const double* __restrict__ sb,
                                                                 double* __restrict__ r) {
  constexpr int N3 = N * N * N, N2 = N * N, NP = N - 1, NP3 = NP * NP * NP, NP2 = NP * NP;
  __shared__ STabSm T;
  __shared__ double X[8][3];
  __shared__ double U[3][N3], Q[3][N3], V[3][N3], T0[N3], T1[N3], R[NP3], TMP[NP3];
  __shared__ double UM[3][N2], UP[3][N2], FA[N2], FT[N2], FR[NP2];
  const int e = blockIdx.x;
  load_tab(tab, T);
  load_cell_vertices(g, verts, e, X);
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) U[i / N3][i % N3] = uh[(size_t)e * 3 * N3 + i];
  for (int i = threadIdx.x; i < NP3; i += blockDim.x) R[i] = 0.0;
  __syncthreads();
  for (int c = 0; c < 3; ++c) sweep3<N, N, false>(T.S, N, U[c], T0, T1, Q[c]);
  // contravariant flux V_m = coef W sum_l J^-1[m][l] uhat_l, tested with d q / d xi_m
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    double Ji[3][3];
    const double W = cell_geom(X, tab, q, N, Ji);
    for (int m = 0; m < 3; ++m) V[m][q] = coef * W * (Ji[m][0] * Q[0][q] + Ji[m][1] * Q[1][q] + Ji[m][2] * Q[2][q]);
  }
  __syncthreads();
  for (int m = 0; m < 3; ++m) {
    sweep<N, N, N, 0, NP, true>(m == 0 ? T.DSp : T.Sp, NP, V[m], T0);
    __syncthreads();
    sweep<NP, N, N, 1, NP, true>(m == 1 ? T.DSp : T.Sp, NP, T0, T1);
    __syncthreads();
    sweep<NP, NP, N, 2, NP, true>(m == 2 ? T.DSp : T.Sp, NP, T1, TMP);
    __syncthreads();
    for (int i = threadIdx.x; i < NP3; i += blockDim.x) R[i] += TMP[i];
    __syncthreads();
  }
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    const int nb = cell_neighbor(g, e, f);
    const bool outflow = nb < 0 && face_bc(g, e, f) != 0;  // velocity Neumann: uhat^+ = uhat^-
    if (nb >= 0 || outflow) {
      for (int c = 0; c < 3; ++c) {
        face_values<N>(U[c], d, s, T, UM[c], FT);
        if (nb >= 0) face_values<N>(uh + (size_t)nb * 3 * N3 + c * N3, d, 1 - s, T, UP[c], FT);
      }
      for (int p = threadIdx.x; p < N2; p += blockDim.x) {
        double Ji[3][3], nrm[3];
        const double Wf = face_geom(X, tab, d, s, p, N, Ji, nrm);
        double an = 0.0;
        for (int c = 0; c < 3; ++c) an += 0.5 * (UM[c][p] + (nb >= 0 ? UP[c][p] : UM[c][p])) * nrm[c];
        FA[p] = -coef * an * Wf;
      }
    } else {
      const int bf = bface_index(g, e, f);
      for (int p = threadIdx.x; p < N2; p += blockDim.x) {
        double Ji[3][3], nrm[3];
        const double Wf = face_geom(X, tab, d, s, p, N, Ji, nrm);
        FA[p] = sb[(size_t)bf * N2 + p] * Wf;
      }
    }
    __syncthreads();
    sweep<N, N, 1, 0, NP, true>(T.Sp, NP, FA, FT);
    __syncthreads();
    sweep<NP, N, 1, 1, NP, true>(T.Sp, NP, FT, FR);
    __syncthreads();
    for (int p = threadIdx.x; p < NP2; p += blockDim.x) R[fnode(d, s, p % NP, p / NP, NP)] += FR[p];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < NP3; i += blockDim.x) r[(size_t)e * NP3 + i] = R[i];
}

// ----------------------------------------------- projection right-hand side
template <int N>
__global__ void __launch_bounds__(kSplitThreads) mproj_rhs_kernel(LevelGeom g, SplitTab tab,
                                                                  const double* __restrict__ verts,
                                                                  const double* __restrict__ p,
                                                                  double* __restrict__ y) {
  constexpr int N3 = N * N * N, N2 = N * N, NP = N - 1, NP3 = NP * NP * NP, NP2 = NP * NP;
  __shared__ STabSm T;
  __shared__ double X[8][3];
  __shared__ double P[NP3], PQ[N3], PJ[3][N3], ACC[N3], T0[N3], T1[N3], OUT[3][N3];
  __shared__ double FA[N2], FB[N2], FT[N2], FR[N2], FC[3][N2];
  const int e = blockIdx.x;
  load_tab(tab, T);
  load_cell_vertices(g, verts, e, X);
  for (int i = threadIdx.x; i < NP3; i += blockDim.x) P[i] = p[(size_t)e * NP3 + i];
  __syncthreads();
  sweep<NP, NP, NP, 0, N, false>(T.Sp, NP, P, T0);
  __syncthreads();
  sweep<N, NP, NP, 1, N, false>(T.Sp, NP, T0, T1);
  __syncthreads();
  sweep<N, N, NP, 2, N, false>(T.Sp, NP, T1, PQ);
  __syncthreads();
  // (div v, p) for v = phi_i e_c: d phi_i / d x_c = sum_m d phi_i / d xi_m J^-1[m][c]
  for (int c = 0; c < 3; ++c) {
    for (int q = threadIdx.x; q < N3; q += blockDim.x) {
      double Ji[3][3];
      const double W = cell_geom(X, tab, q, N, Ji);
      for (int m = 0; m < 3; ++m) PJ[m][q] = W * PQ[q] * Ji[m][c];
      ACC[q] = 0.0;
    }
    __syncthreads();
    for (int m = 0; m < 3; ++m) {
      sweep_dir<N, true>(m, T.Dg, PJ[m], T0);
      __syncthreads();
      for (int q = threadIdx.x; q < N3; q += blockDim.x) ACC[q] += T0[q];
      __syncthreads();
    }
    sweep3<N, N, true>(T.S, N, ACC, T0, T1, OUT[c]);
  }
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    const int nb = cell_neighbor(g, e, f);
    if (nb < 0 && face_bc(g, e, f) != 0) continue;  // pressure Dirichlet, datum 0: {{p}} = 0
    for (int q = threadIdx.x; q < NP2; q += blockDim.x) {
      FA[q] = P[fnode(d, s, q % NP, q / NP, NP)];
      FB[q] = nb >= 0 ? p[(size_t)nb * NP3 + fnode(d, 1 - s, q % NP, q / NP, NP)] : FA[q];
    }
    __syncthreads();
    sweep<NP, NP, 1, 0, N, false>(T.Sp, NP, FA, FT);
    __syncthreads();
    sweep<N, NP, 1, 1, N, false>(T.Sp, NP, FT, FA);
    __syncthreads();
    sweep<NP, NP, 1, 0, N, false>(T.Sp, NP, FB, FT);
    __syncthreads();
    sweep<N, NP, 1, 1, N, false>(T.Sp, NP, FT, FB);
    __syncthreads();
    for (int q = threadIdx.x; q < N2; q += blockDim.x) {
      double Ji[3][3], nrm[3];
      const double Wf = face_geom(X, tab, d, s, q, N, Ji, nrm);
      const double pavg = 0.5 * (FA[q] + FB[q]);
      for (int c = 0; c < 3; ++c) FC[c][q] = -pavg * nrm[c] * Wf;
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) face_values_t<N>(FC[c], d, s, T, OUT[c], FT, FR);
  }
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) y[(size_t)e * 3 * N3 + i] = OUT[i / N3][i % N3];
}

// ---------------------------------------- viscous wall data (right-hand side)
// D_a = -(2 nu eps(phi_a) n, g) + (2 tau, phi_a.g + (phi_a.n)(g.n)) over Dirichlet
// faces; for phi_a = phi_i e_c: (2 nu eps(phi_a) n).g = nu (g_c grad phi_i.n + n_c grad phi_i.g)
template <int N>
__global__ void __launch_bounds__(kSplitThreads) mvisc_dir_kernel(LevelGeom g, SplitTab tab, Wall wall,
                                                                  const double* __restrict__ verts,
                                                                  const double* __restrict__ lam,
                                                                  const double* __restrict__ nu_face,
                                                                  double* __restrict__ y) {
  constexpr int N3 = N * N * N, N2 = N * N;
  __shared__ STabSm T;
  __shared__ double X[8][3];
  __shared__ double OUT[3][N3], CF[3][4 * N2], SC[5 * N2];
  const int e = blockIdx.x;
  load_tab(tab, T);
  load_cell_vertices(g, verts, e, X);
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) OUT[i / N3][i % N3] = 0.0;
  __syncthreads();
  const double lam_e = lam[e];
  for (int f = 0; f < 6; ++f) {
    if (cell_neighbor(g, e, f) >= 0 || face_bc(g, e, f) != 0) continue;
    if (!wall.pts) {
      const double* gc = wall.g[boundary_id(g, e, f)];
      if (gc[0] == 0.0 && gc[1] == 0.0 && gc[2] == 0.0) continue;
    }
    const int d = f >> 1, s = f & 1;
    int t1, t2;
    face_dirs(d, &t1, &t2);
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      double Ji[3][3], nrm[3];
      const double Wf = face_geom(X, tab, d, s, p, N, Ji, nrm);
      const double nu = nu_face[((size_t)e * 6 + f) * N2 + p];
      const double tau = g.cip * (double)(N * N) * lam_e * nu;
      double gv[3];
      for (int j = 0; j < 3; ++j) gv[j] = wall_val(wall, g, e, f, p, j, N2);
      const double gn = gv[0] * nrm[0] + gv[1] * nrm[1] + gv[2] * nrm[2];
      for (int c = 0; c < 3; ++c) {
        double cv[3], R[3];
        for (int l = 0; l < 3; ++l) cv[l] = -Wf * nu * (gv[c] * nrm[l] + nrm[c] * gv[l]);
        for (int m = 0; m < 3; ++m) R[m] = cv[0] * Ji[m][0] + cv[1] * Ji[m][1] + cv[2] * Ji[m][2];
        CF[c][p] = 2.0 * tau * Wf * (gv[c] + nrm[c] * gn);
        CF[c][N2 + p] = R[d];
        CF[c][2 * N2 + p] = R[t1];
        CF[c][3 * N2 + p] = R[t2];
      }
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) face_eval_t<N>(CF[c], d, s, T, OUT[c], SC);
  }
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) y[(size_t)e * 3 * N3 + i] = OUT[i / N3][i % N3];
}

// ------------------------------------------------------------------- CFL
template <int N>
__global__ void __launch_bounds__(kSplitThreads) mcfl_kernel(LevelGeom g, SplitTab tab,
                                                             const double* __restrict__ verts,
                                                             const double* __restrict__ u,
                                                             unsigned long long* __restrict__ vmax_bits) {
  constexpr int N3 = N * N * N;
  __shared__ STabSm T;
  __shared__ double X[8][3];
  __shared__ double U[3][N3], Q[3][N3], T0[N3], T1[N3];
  __shared__ double red[kSplitThreads];
  const int e = blockIdx.x;
  load_tab(tab, T);
  load_cell_vertices(g, verts, e, X);
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) U[i / N3][i % N3] = u[(size_t)e * 3 * N3 + i];
  __syncthreads();
  for (int c = 0; c < 3; ++c) sweep3<N, N, false>(T.S, N, U[c], T0, T1, Q[c]);
  double m = 0.0;
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    double Ji[3][3];
    cell_geom(X, tab, q, N, Ji);
    double v[3];
    for (int k = 0; k < 3; ++k) v[k] = Ji[k][0] * Q[0][q] + Ji[k][1] * Q[1][q] + Ji[k][2] * Q[2][q];
    m = fmax(m, sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(vmax_bits, (unsigned long long)__double_as_longlong(red[0]));
}

// ------------------------------------------------------------ cell mass
template <int N>
__global__ void __launch_bounds__(kSplitThreads) mmass_kernel(LevelGeom g, SplitTab tab, int ncomp,
                                                              const double* __restrict__ verts, double coeff,
                                                              bool inverse, const double* __restrict__ x,
                                                              double* __restrict__ y) {
  constexpr int N3 = N * N * N;
  __shared__ STabSm T;
  __shared__ double X[8][3];
  __shared__ double SI[kMaxN * kMaxN];
  __shared__ double A[N3], B[N3], C[N3], WQ[N3];
  const int e = blockIdx.x;
  load_tab(tab, T);
  load_cell_vertices(g, verts, e, X);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) SI[i] = tab.Sinv[i];
  __syncthreads();
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    double Ji[3][3];
    WQ[q] = coeff * cell_geom(X, tab, q, N, Ji);
  }
  for (int c = 0; c < ncomp; ++c) {
    const size_t base = ((size_t)e * ncomp + c) * N3;
    for (int i = threadIdx.x; i < N3; i += blockDim.x) A[i] = x[base + i];
    __syncthreads();
    if (!inverse) {  // S^T (coeff W) S x
      sweep3<N, N, false>(T.S, N, A, B, C, A);
      for (int q = threadIdx.x; q < N3; q += blockDim.x) A[q] *= WQ[q];
      __syncthreads();
      sweep3<N, N, true>(T.S, N, A, B, C, A);
    } else {  // S^-1 (coeff W)^-1 S^-T x
      sweep3<N, N, true>(SI, N, A, B, C, A);
      for (int q = threadIdx.x; q < N3; q += blockDim.x) A[q] /= WQ[q];
      __syncthreads();
      sweep3<N, N, false>(SI, N, A, B, C, A);
    }
    for (int i = threadIdx.x; i < N3; i += blockDim.x) y[base + i] = A[i];
    __syncthreads();
  }
}

// positions of the Gauss points of every boundary face, [nbf][n^2][3]
template <int N>
__global__ void mbpoints_kernel(LevelGeom g, SplitTab tab, const double* __restrict__ verts, int nbf,
                                double* __restrict__ xyz) {
  __shared__ double X[8][3];
  const int b = blockIdx.x;
  int e, f;
  bface_cell(g, b, &e, &f);
  load_cell_vertices(g, verts, e, X);
  __syncthreads();
  const int d = f >> 1, s = f & 1;
  for (int p = threadIdx.x; p < N * N; p += blockDim.x) {
    double Ji[3][3], nrm[3], pos[3];
    face_geom(X, tab, d, s, p, N, Ji, nrm, pos);
    for (int c = 0; c < 3; ++c) xyz[((size_t)b * N * N + p) * 3 + c] = pos[c];
  }
}

}  // namespace

#define SIPG_MSPLIT_DISPATCH(NN, CALL)              \
  switch (NN) {                                     \
    case 3: { constexpr int N = 3; CALL; break; }   \
    case 4: { constexpr int N = 4; CALL; break; }   \
    case 5: { constexpr int N = 5; CALL; break; }   \
    case 6: { constexpr int N = 6; CALL; break; }   \
    default: return cudaErrorInvalidValue;          \
  }

cudaError_t launch_mapped_convective(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                     const WallArg& wall_g, const double* u, double* y, cudaStream_t st) {
  const Wall w = make_wall(wall_g);
  if (g.ncells == 0) return cudaSuccess;
  SIPG_MSPLIT_DISPATCH(n, (mconv_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, w, verts, u, y)));
  return cudaGetLastError();
}

cudaError_t launch_mapped_ppe_boundary(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                       const WallArg& wall_g, const PpeBndArgs& a, const RheologyDev& rh,
                                       const double* u0, const double* u1, double* sb, cudaStream_t st) {
  const Wall w = make_wall(wall_g);
  MPpeBnd pb{};
  pb.a = a;
  pb.rh = rh;
  const int nbf = n_wall_faces(g);
  if (nbf == 0) return cudaSuccess;
  SIPG_MSPLIT_DISPATCH(n, (mppe_bnd_kernel<N><<<nbf, kSplitThreads, 0, st>>>(g, tab, w, pb, verts, u0, u1, sb)));
  return cudaGetLastError();
}

cudaError_t launch_mapped_ppe_rhs(int n, const LevelGeom& g, const SplitTab& tab, const double* verts, double coef,
                                  const double* uhat, const double* sb, double* r, cudaStream_t st) {
  if (g.ncells == 0) return cudaSuccess;
  SIPG_MSPLIT_DISPATCH(n, (mppe_rhs_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, coef, verts, uhat, sb, r)));
  return cudaGetLastError();
}

cudaError_t launch_mapped_projection_rhs(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                         const double* p, double* y, cudaStream_t st) {
  if (g.ncells == 0) return cudaSuccess;
  SIPG_MSPLIT_DISPATCH(n, (mproj_rhs_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, verts, p, y)));
  return cudaGetLastError();
}

cudaError_t launch_mapped_viscous_wall_rhs(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                           const double* lam, const WallArg& wall_g, const double* nu_face,
                                           double* y, cudaStream_t st) {
  const Wall w = make_wall(wall_g);
  if (g.ncells == 0) return cudaSuccess;
  SIPG_MSPLIT_DISPATCH(n, (mvisc_dir_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, w, verts, lam, nu_face,
                                                                                    y)));
  return cudaGetLastError();
}

cudaError_t launch_mapped_cfl_max(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                  const double* u, unsigned long long* vmax_bits, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(vmax_bits, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess || g.ncells == 0) return e;
  SIPG_MSPLIT_DISPATCH(n, (mcfl_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, verts, u, vmax_bits)));
  return cudaGetLastError();
}

cudaError_t launch_mapped_mass(int n, int ncomp, const LevelGeom& g, const SplitTab& tab, const double* verts,
                               double coeff, bool inverse, const double* x, double* y, cudaStream_t st) {
  if (g.ncells == 0) return cudaSuccess;
  switch (n) {
    case 2: mmass_kernel<2><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, ncomp, verts, coeff, inverse, x, y); break;
    case 3: mmass_kernel<3><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, ncomp, verts, coeff, inverse, x, y); break;
    case 4: mmass_kernel<4><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, ncomp, verts, coeff, inverse, x, y); break;
    case 5: mmass_kernel<5><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, ncomp, verts, coeff, inverse, x, y); break;
    case 6: mmass_kernel<6><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, ncomp, verts, coeff, inverse, x, y); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_mapped_boundary_points(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                          double* xyz, cudaStream_t st) {
  const int nbf = n_wall_faces(g);
  if (nbf == 0) return cudaSuccess;
  SIPG_MSPLIT_DISPATCH(n, (mbpoints_kernel<N><<<nbf, 64, 0, st>>>(g, tab, verts, nbf, xyz)));
  return cudaGetLastError();
}

}  // namespace sipg
