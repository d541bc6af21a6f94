// Forms of one step of the projection scheme on affine grids (the box, the
// backward-facing-step channel; Sec. 3.2 / 5.1, Alg. 1),
// convective term explicit:
//   conv_kernel       C_a = c_h(phi_a, u; u), Eq. (convective_term_weak), upwind flux,
//                     mirror principle on Dirichlet walls
//   ppe_bnd_kernel    h_p - (gamma0/dt) g_uhat.n at the Gauss points of every
//                     wall face, Eqs. (pressure_Neumann_BC), (guhat_consistent_BC)
//   ppe_rhs_kernel    (gamma0/dt)[(grad q, uhat) - (q, {{uhat}}.n)] with the wall
//                     datum above on Dirichlet faces and uhat^+ = uhat^- on
//                     outflow (velocity Neumann) faces, Eq. (pressure_step_weak)
//   proj_rhs_kernel   (div v, p) - (v, {{p}} n), Eq. (projection_step_weak)
//   visc_dir_kernel   Dirichlet wall-data terms of the SIPG viscous form (mirror
//                     u^+ = -u^- + 2g) for the viscous step's right-hand side
//   cfl_kernel        max over Gauss points of |J^-1 u|, Eq. (CFL_timestep_selection)
//
// All FP64, one CTA per cell (or per wall face), one thread per tensor entry in
// each 1D sweep; every CTA writes only its own rows (no atomics except the max
// of the CFL reduction, which is order independent). Fields given at the n^3
// Gauss points of a cell are the values of a Q_k polynomial there (n = k+1
// points per direction determine it), so traces and derivatives of such a
// field are taken exactly with the Lagrange basis on the Gauss points; in
// particular the element-local L2 projection onto Q_k of point values at the
// Gauss points is the polynomial interpolating them (M1^-1 S^T W = S^-1).
#include "kernels.cuh"
#include "sweeps.cuh"

#include <algorithm>

namespace sipg {
namespace {

using namespace sweeps;

// --------------------------------------------------------------- convective
template <int N>
__global__ void __launch_bounds__(kSplitThreads) conv_kernel(LevelGeom g, SplitTab tab, Wall wall,
                                                             const double* __restrict__ u, double* __restrict__ y) {
  constexpr int N3 = N * N * N, N2 = N * N;
  __shared__ STabSm T;
  __shared__ double U[3][N3], Q[3][N3], G[3][3][N3], CV[3][N3], T0[N3], T1[N3], OUT[3][N3];
  __shared__ double UM[3][N2], UP[3][N2], FT[N2], FL[3][N2], FR[N2];
  const int e = blockIdx.x;
  load_tab(tab, T);
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) U[i / N3][i % N3] = u[(size_t)e * 3 * N3 + i];
  __syncthreads();
  for (int c = 0; c < 3; ++c) sweep3<N, N, false>(T.S, N, U[c], T0, T1, Q[c]);
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l < 3; ++l) sweep_dir<N, false>(l, T.Dg, Q[c], G[c][l]);
  __syncthreads();
  const double detJ = g.h[0] * g.h[1] * g.h[2];
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    const double w = cell_weight(T, q, N, detJ);
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int l = 0; l < 3; ++l) acc += Q[l][q] * G[c][l][q] * g.ih[l];
      CV[c][q] = w * acc;
    }
  }
  __syncthreads();
  for (int c = 0; c < 3; ++c) sweep3<N, N, true>(T.S, N, CV[c], T0, T1, OUT[c]);
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    int t1, t2;
    face_dirs(d, &t1, &t2);
    const double nd = 2.0 * s - 1.0;
    const int nb = cell_neighbor(g, e, f);
    for (int i = threadIdx.x; i < 3 * N2; i += blockDim.x) {
      const int c = i / N2, p = i % N2;
      FL[c][p] = U[c][fnode(d, s, p % N, p / N, N)];
      if (nb >= 0) CV[c][p] = u[(size_t)nb * 3 * N3 + c * N3 + fnode(d, 1 - s, p % N, p / N, N)];
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
      sweep<N, N, 1, 0, N, false>(T.S, N, FL[c], FT);
      __syncthreads();
      sweep<N, N, 1, 1, N, false>(T.S, N, FT, UM[c]);
      __syncthreads();
      if (nb >= 0) {
        sweep<N, N, 1, 0, N, false>(T.S, N, CV[c], FT);
        __syncthreads();
        sweep<N, N, 1, 1, N, false>(T.S, N, FT, UP[c]);
        __syncthreads();
      }
    }
    const double area = g.h[t1] * g.h[t2];
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      double um[3], up[3];
      for (int c = 0; c < 3; ++c) {
        um[c] = UM[c][p];
        up[c] = nb >= 0 ? UP[c][p] : (face_bc(g, e, f) == 0 ? -um[c] + 2.0 * wall_val(wall, g, e, f, p, c, N2) : um[c]);
      }
      const double wn = 0.5 * (um[d] + up[d]) * nd;
      const double sg = wn > 0.0 ? 1.0 : (wn < 0.0 ? -1.0 : 0.0);
      const double w = T.gw[p % N] * T.gw[p / N] * area;
      for (int c = 0; c < 3; ++c) FL[c][p] = w * wn * 0.5 * (1.0 - sg) * (up[c] - um[c]);
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
      sweep<N, N, 1, 0, N, true>(T.S, N, FL[c], FT);
      __syncthreads();
      sweep<N, N, 1, 1, N, true>(T.S, N, FT, FR);
      __syncthreads();
      for (int p = threadIdx.x; p < N2; p += blockDim.x) OUT[c][fnode(d, s, p % N, p / N, N)] += FR[p];
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) y[(size_t)e * 3 * N3 + i] = OUT[i / N3][i % N3];
}

// --------------------------------------------- linearised convective term
// y = sum_e c_h(phi, u; w) for a fixed transport velocity w (linear in u; the
// alpha_c = 1, u* = u# term of Eq. viscous_step_weak). Walls: u^+ = -u^- + 2 gu,
// w^+ = -w^- + 2 gw. With gu = 0 this is the homogeneous operator of the
// Krylov solve; with u = 0 it is the wall-data part (right-hand side, negated).
template <int N>
__global__ void __launch_bounds__(kSplitThreads) conv_lin_kernel(LevelGeom g, SplitTab tab, Wall wall_w, Wall wall_u,
                                                                 const double* __restrict__ w,
                                                                 const double* __restrict__ u,
                                                                 double* __restrict__ y) {
  constexpr int N3 = N * N * N, N2 = N * N;
  __shared__ STabSm T;
  __shared__ double U[3][N3], Q[3][N3], G[3][3][N3], CV[3][N3], T0[N3], T1[N3], OUT[3][N3];
  __shared__ double UM[3][N2], UP[3][N2], WM[3][N2], WP[3][N2], FT[N2], FL[3][N2], FR[N2];
  const int e = blockIdx.x;
  load_tab(tab, T);
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) {
    U[i / N3][i % N3] = u[(size_t)e * 3 * N3 + i];
    CV[i / N3][i % N3] = w[(size_t)e * 3 * N3 + i];
  }
  __syncthreads();
  for (int c = 0; c < 3; ++c) sweep3<N, N, false>(T.S, N, U[c], T0, T1, Q[c]);
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l < 3; ++l) sweep_dir<N, false>(l, T.Dg, Q[c], G[c][l]);
  __syncthreads();
  for (int c = 0; c < 3; ++c) sweep3<N, N, false>(T.S, N, CV[c], T0, T1, Q[c]);  // w at the Gauss points
  const double detJ = g.h[0] * g.h[1] * g.h[2];
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    const double wq = cell_weight(T, q, N, detJ);
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int l = 0; l < 3; ++l) acc += Q[l][q] * G[c][l][q] * g.ih[l];
      CV[c][q] = wq * acc;
    }
  }
  __syncthreads();
  for (int c = 0; c < 3; ++c) sweep3<N, N, true>(T.S, N, CV[c], T0, T1, OUT[c]);
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    int t1, t2;
    face_dirs(d, &t1, &t2);
    const double nd = 2.0 * s - 1.0;
    const int nb = cell_neighbor(g, e, f);
    if (nb < 0 && face_bc(g, e, f) != 0) continue;  // Neumann: u^+ = u^-, w^+ = w^-: no flux
    // face nodes: own u, own w, neighbour u, neighbour w (in Q as scratch)
    for (int i = threadIdx.x; i < 3 * N2; i += blockDim.x) {
      const int c = i / N2, p = i % N2;
      const int own = fnode(d, s, p % N, p / N, N);
      Q[0][i] = U[c][own];
      Q[1][i] = w[(size_t)e * 3 * N3 + c * N3 + own];
      if (nb >= 0) {
        const int oth = fnode(d, 1 - s, p % N, p / N, N);
        Q[2][i] = u[(size_t)nb * 3 * N3 + c * N3 + oth];
        CV[0][i] = w[(size_t)nb * 3 * N3 + c * N3 + oth];
      }
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
      sweep<N, N, 1, 0, N, false>(T.S, N, Q[0] + c * N2, FT);
      __syncthreads();
      sweep<N, N, 1, 1, N, false>(T.S, N, FT, UM[c]);
      __syncthreads();
      sweep<N, N, 1, 0, N, false>(T.S, N, Q[1] + c * N2, FT);
      __syncthreads();
      sweep<N, N, 1, 1, N, false>(T.S, N, FT, WM[c]);
      __syncthreads();
      if (nb >= 0) {
        sweep<N, N, 1, 0, N, false>(T.S, N, Q[2] + c * N2, FT);
        __syncthreads();
        sweep<N, N, 1, 1, N, false>(T.S, N, FT, UP[c]);
        __syncthreads();
        sweep<N, N, 1, 0, N, false>(T.S, N, CV[0] + c * N2, FT);
        __syncthreads();
        sweep<N, N, 1, 1, N, false>(T.S, N, FT, WP[c]);
        __syncthreads();
      }
    }
    const double area = g.h[t1] * g.h[t2];
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      double um[3], up[3], wm, wp;
      for (int c = 0; c < 3; ++c) {
        um[c] = UM[c][p];
        up[c] = nb >= 0 ? UP[c][p] : -um[c] + 2.0 * wall_val(wall_u, g, e, f, p, c, N2);
      }
      wm = WM[d][p];
      wp = nb >= 0 ? WP[d][p] : -wm + 2.0 * wall_val(wall_w, g, e, f, p, d, N2);
      const double wn = 0.5 * (wm + wp) * nd;
      const double sg = wn > 0.0 ? 1.0 : (wn < 0.0 ? -1.0 : 0.0);
      const double wt = T.gw[p % N] * T.gw[p / N] * area;
      for (int c = 0; c < 3; ++c) FL[c][p] = wt * wn * 0.5 * (1.0 - sg) * (up[c] - um[c]);
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
      sweep<N, N, 1, 0, N, true>(T.S, N, FL[c], FT);
      __syncthreads();
      sweep<N, N, 1, 1, N, true>(T.S, N, FT, FR);
      __syncthreads();
      for (int p = threadIdx.x; p < N2; p += blockDim.x) OUT[c][fnode(d, s, p % N, p / N, N)] += FR[p];
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) y[(size_t)e * 3 * N3 + i] = OUT[i / N3][i % N3];
}

// ----------------------------------------------------- PPE wall datum
// h_p - (gamma0/dt) g_uhat.n = sum_{i<m} (beta_i - betabar_i) n.(u^{n-i}.grad)u^{n-i}
//     - nu^dd n.curl omega^dd + 2 n.(eps(u^dd) grad nu^dd) - (gamma0/dt) g.n
// (n.b cancels between h_p and g_uhat; sum_i alpha_i = gamma0 for BDF).
struct PpeBnd {
  PpeBndArgs a;
  RheologyDev rh;  // constant or Carreau-Yasuda
};

__device__ __forceinline__ double eta_of(const RheologyDev& r, const double G[3][3]) {
  if (r.law == 0) return r.nu;
  double ee = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      const double e = 0.5 * (G[k][l] + G[l][k]);
      ee += e * e;
    }
  const double gdot = sqrt(2.0 * ee);
  return r.eta_inf + (r.eta0 - r.eta_inf) * pow(r.kappa + pow(r.lambda * gdot, r.a), (r.b - 1.0) / r.a);
}

template <int N>
__global__ void __launch_bounds__(kSplitThreads) ppe_bnd_kernel(LevelGeom g, SplitTab tab, Wall wall, PpeBnd pb,
                                                                const double* __restrict__ u0,
                                                                const double* __restrict__ u1,
                                                                double* __restrict__ sb) {
  constexpr int N3 = N * N * N, N2 = N * N;
  __shared__ STabSm T;
  __shared__ double U[3][N3], Q[3][N3], G[3][3][N3], T0[N3], T1[N3], W3[3][N3];
  __shared__ double TR[12][N2], ACC[N2];
  // the wall face: cell e, face f
  int e, f;
  bface_cell(g, blockIdx.x, &e, &f);
  if (face_bc(g, e, f) != 0) {  // velocity Neumann (pressure Dirichlet): no datum
    for (int p = threadIdx.x; p < N2; p += blockDim.x) sb[(size_t)blockIdx.x * N2 + p] = 0.0;
    return;
  }
  const int d = f >> 1, s = f & 1;
  int t1, t2;
  face_dirs(d, &t1, &t2);
  const double nd = 2.0 * s - 1.0;
  load_tab(tab, T);
  for (int p = threadIdx.x; p < N2; p += blockDim.x) ACC[p] = pb.a.gn_coef * wall_val(wall, g, e, f, p, d, N2) * nd;
  __syncthreads();
  // convective terms: n.(u.grad)u of each history, weight beta_i - betabar_i
  for (int h = 0; h < pb.a.n_hist; ++h) {
    const double* uh = h == 0 ? u0 : u1;
    if (pb.a.wconv[h] == 0.0) continue;
    for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) U[i / N3][i % N3] = uh[(size_t)e * 3 * N3 + i];
    __syncthreads();
    for (int c = 0; c < 3; ++c) sweep3<N, N, false>(T.S, N, U[c], T0, T1, Q[c]);
    for (int l = 0; l < 3; ++l) sweep_dir<N, false>(l, T.Dg, Q[d], G[d][l]);
    __syncthreads();
    for (int c = 0; c < 3; ++c) trace<N>(Q[c], T.lg[s], d, TR[c]);
    for (int l = 0; l < 3; ++l) trace<N>(G[d][l], T.lg[s], d, TR[3 + l]);
    __syncthreads();
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      double cv = 0.0;
      for (int l = 0; l < 3; ++l) cv += TR[l][p] * TR[3 + l][p] * g.ih[l];
      ACC[p] += pb.a.wconv[h] * nd * cv;
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
      for (int l = 0; l < 3; ++l) sweep_dir<N, false>(l, T.Dg, Q[c], G[c][l]);
    __syncthreads();
    // vorticity and viscosity at the Gauss points (their L2 projections onto Q_k)
    for (int q = threadIdx.x; q < N3; q += blockDim.x) {
      double Gq[3][3];
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) Gq[k][l] = G[k][l][q] * g.ih[l];
      W3[0][q] = Gq[2][1] - Gq[1][2];
      W3[1][q] = Gq[0][2] - Gq[2][0];
      W3[2][q] = Gq[1][0] - Gq[0][1];
      T0[q] = eta_of(pb.rh, Gq);
    }
    __syncthreads();
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    // traces: omega_{d1}, omega_{d2}, nu, d nu / dn, and the 9 gradient entries
    trace<N>(W3[d1], T.lg[s], d, TR[0]);
    trace<N>(W3[d2], T.lg[s], d, TR[1]);
    trace<N>(T0, T.lg[s], d, TR[2]);
    trace<N>(T0, T.dlg[s], d, TR[3]);
    __syncthreads();
    // tangential derivatives on the face Gauss grid: d/dt1 of a field = Dg along a
    // (TR[4..7]: d omega_{d1}/dt1, /dt2, d omega_{d2}/dt1, /dt2; TR[8], TR[9]: d nu/dt1, /dt2)
    sweep<N, N, 1, 0, N, false>(T.Dg, N, TR[0], TR[4]);
    sweep<N, N, 1, 1, N, false>(T.Dg, N, TR[0], TR[5]);
    sweep<N, N, 1, 0, N, false>(T.Dg, N, TR[1], TR[6]);
    sweep<N, N, 1, 1, N, false>(T.Dg, N, TR[1], TR[7]);
    sweep<N, N, 1, 0, N, false>(T.Dg, N, TR[2], TR[8]);
    sweep<N, N, 1, 1, N, false>(T.Dg, N, TR[2], TR[9]);
    __syncthreads();
    // d/d x_{d1} and d/d x_{d2} in terms of t1 < t2
    const bool d1_is_t1 = d1 == t1;
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      const double dw2_dd1 = (d1_is_t1 ? TR[6][p] : TR[7][p]) * g.ih[d1];
      const double dw1_dd2 = (d1_is_t1 ? TR[5][p] : TR[4][p]) * g.ih[d2];
      const double curl_d = dw2_dd1 - dw1_dd2;
      double gradnu[3];
      gradnu[d] = TR[3][p] * g.ih[d];
      gradnu[t1] = TR[8][p] * g.ih[t1];
      gradnu[t2] = TR[9][p] * g.ih[t2];
      T1[p] = curl_d;
      for (int l = 0; l < 3; ++l) Q[0][p * 3 + l] = gradnu[l];  // Q is free now: grad nu at face points
    }
    __syncthreads();
    // gradient of u^dd at the face points (traces of the Gauss-point gradients)
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) trace<N>(G[k][l], T.lg[s], d, W3[0] + (k * 3 + l) * N2);
    __syncthreads();
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      double Gf[3][3];
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) Gf[k][l] = W3[0][(k * 3 + l) * N2 + p] * g.ih[l];
      const double nu = eta_of(pb.rh, Gf);
      double epsgrad = 0.0;
      for (int l = 0; l < 3; ++l) epsgrad += 0.5 * (Gf[d][l] + Gf[l][d]) * Q[0][p * 3 + l];
      ACC[p] += -nu * nd * T1[p] + 2.0 * nd * epsgrad;
    }
    __syncthreads();
  }
  for (int p = threadIdx.x; p < N2; p += blockDim.x) sb[(size_t)blockIdx.x * N2 + p] = ACC[p];
}

// ------------------------------------------------------ PPE right-hand side
template <int N>
__global__ void __launch_bounds__(kSplitThreads) ppe_rhs_kernel(LevelGeom g, SplitTab tab, double coef,
                                                                const double* __restrict__ uh,
                                                                const double* __restrict__ sb,
                                                                double* __restrict__ r) {
  constexpr int N3 = N * N * N, N2 = N * N, NP = N - 1, NP3 = NP * NP * NP, NP2 = NP * NP;
  __shared__ STabSm T;
  __shared__ double U[3][N3], Q[N3], T0[N3], T1[N3], R[NP3], TMP[NP3];
  __shared__ double FA[N2], FB[N2], FT[N2], FR[NP2];
  const int e = blockIdx.x;
  load_tab(tab, T);
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) U[i / N3][i % N3] = uh[(size_t)e * 3 * N3 + i];
  for (int i = threadIdx.x; i < NP3; i += blockDim.x) R[i] = 0.0;
  __syncthreads();
  const double detJ = g.h[0] * g.h[1] * g.h[2];
  for (int l = 0; l < 3; ++l) {
    sweep3<N, N, false>(T.S, N, U[l], T0, T1, Q);
    for (int q = threadIdx.x; q < N3; q += blockDim.x) Q[q] *= coef * cell_weight(T, q, N, detJ) * g.ih[l];
    __syncthreads();
    // (grad q)_l: derivative of the pressure basis along l, values along the others
    sweep<N, N, N, 0, NP, true>(l == 0 ? T.DSp : T.Sp, NP, Q, T0);
    __syncthreads();
    sweep<NP, N, N, 1, NP, true>(l == 1 ? T.DSp : T.Sp, NP, T0, T1);
    __syncthreads();
    sweep<NP, NP, N, 2, NP, true>(l == 2 ? T.DSp : T.Sp, NP, T1, TMP);
    __syncthreads();
    for (int i = threadIdx.x; i < NP3; i += blockDim.x) R[i] += TMP[i];
    __syncthreads();
  }
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    int t1, t2;
    face_dirs(d, &t1, &t2);
    const double nd = 2.0 * s - 1.0;
    const int nb = cell_neighbor(g, e, f);
    // velocity Neumann (outflow): uhat^+ = uhat^-, so {{uhat}}.n = uhat^-.n
    const bool outflow = nb < 0 && face_bc(g, e, f) != 0;
    const double area = g.h[t1] * g.h[t2];
    if (nb >= 0 || outflow) {
      for (int p = threadIdx.x; p < N2; p += blockDim.x) {
        FA[p] = U[d][fnode(d, s, p % N, p / N, N)];
        FB[p] = outflow ? FA[p] : uh[(size_t)nb * 3 * N3 + d * N3 + fnode(d, 1 - s, p % N, p / N, N)];
      }
      __syncthreads();
      sweep<N, N, 1, 0, N, false>(T.S, N, FA, FT);
      __syncthreads();
      sweep<N, N, 1, 1, N, false>(T.S, N, FT, FA);
      __syncthreads();
      sweep<N, N, 1, 0, N, false>(T.S, N, FB, FT);
      __syncthreads();
      sweep<N, N, 1, 1, N, false>(T.S, N, FT, FB);
      __syncthreads();
      for (int p = threadIdx.x; p < N2; p += blockDim.x)
        FA[p] = -coef * 0.5 * (FA[p] + FB[p]) * nd * T.gw[p % N] * T.gw[p / N] * area;
    } else {
      const int bf = bface_index(g, e, f);
      for (int p = threadIdx.x; p < N2; p += blockDim.x)
        FA[p] = sb[(size_t)bf * N2 + p] * T.gw[p % N] * T.gw[p / N] * area;
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
__global__ void __launch_bounds__(kSplitThreads) proj_rhs_kernel(LevelGeom g, SplitTab tab,
                                                                 const double* __restrict__ p,
                                                                 double* __restrict__ y) {
  constexpr int N3 = N * N * N, N2 = N * N, NP = N - 1, NP3 = NP * NP * NP, NP2 = NP * NP;
  __shared__ STabSm T;
  __shared__ double P[NP3], PQ[N3], T0[N3], T1[N3], OUT[3][N3];
  __shared__ double FA[N2], FB[N2], FT[N2], FR[N2];
  const int e = blockIdx.x;
  load_tab(tab, T);
  for (int i = threadIdx.x; i < NP3; i += blockDim.x) P[i] = p[(size_t)e * NP3 + i];
  __syncthreads();
  sweep<NP, NP, NP, 0, N, false>(T.Sp, NP, P, T0);
  __syncthreads();
  sweep<N, NP, NP, 1, N, false>(T.Sp, NP, T0, T1);
  __syncthreads();
  sweep<N, N, NP, 2, N, false>(T.Sp, NP, T1, PQ);
  __syncthreads();
  const double detJ = g.h[0] * g.h[1] * g.h[2];
  for (int q = threadIdx.x; q < N3; q += blockDim.x) PQ[q] *= cell_weight(T, q, N, detJ);
  __syncthreads();
  for (int c = 0; c < 3; ++c) {
    // (div v, p) for v = phi_i e_c: d phi_i / d x_c
    sweep<N, N, N, 0, N, true>(c == 0 ? T.DS : T.S, N, PQ, T0);
    __syncthreads();
    sweep<N, N, N, 1, N, true>(c == 1 ? T.DS : T.S, N, T0, T1);
    __syncthreads();
    sweep<N, N, N, 2, N, true>(c == 2 ? T.DS : T.S, N, T1, OUT[c]);
    __syncthreads();
    for (int i = threadIdx.x; i < N3; i += blockDim.x) OUT[c][i] *= g.ih[c];
    __syncthreads();
  }
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    int t1, t2;
    face_dirs(d, &t1, &t2);
    const double nd = 2.0 * s - 1.0;
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
    const double area = g.h[t1] * g.h[t2];
    for (int q = threadIdx.x; q < N2; q += blockDim.x)
      FA[q] = -0.5 * (FA[q] + FB[q]) * nd * T.gw[q % N] * T.gw[q / N] * area;
    __syncthreads();
    sweep<N, N, 1, 0, N, true>(T.S, N, FA, FT);
    __syncthreads();
    sweep<N, N, 1, 1, N, true>(T.S, N, FT, FR);
    __syncthreads();
    for (int q = threadIdx.x; q < N2; q += blockDim.x) OUT[d][fnode(d, s, q % N, q / N, N)] += FR[q];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) y[(size_t)e * 3 * N3 + i] = OUT[i / N3][i % N3];
}

// ---------------------------------------- viscous wall data (right-hand side)
template <int N>
__global__ void __launch_bounds__(kSplitThreads) visc_dir_kernel(LevelGeom g, SplitTab tab, Wall wall,
                                                                 const double* __restrict__ nu_face,
                                                                 double* __restrict__ y) {
  constexpr int N3 = N * N * N, N2 = N * N;
  __shared__ STabSm T;
  __shared__ double OUT[3][N3], CA[N2], CB[N2], CC[N2], CE[N2], FT[N2], FR[N2];
  const int e = blockIdx.x;
  load_tab(tab, T);
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) OUT[i / N3][i % N3] = 0.0;
  __syncthreads();
  const double lam = penalty_lambda(g, e);
  for (int f = 0; f < 6; ++f) {
    if (cell_neighbor(g, e, f) >= 0 || face_bc(g, e, f) != 0) continue;
    if (!wall.pts) {
      const double* gc = wall.g[boundary_id(g, e, f)];
      if (gc[0] == 0.0 && gc[1] == 0.0 && gc[2] == 0.0) continue;
    }
    const int d = f >> 1, s = f & 1;
    int t1, t2;
    face_dirs(d, &t1, &t2);
    const double nd = 2.0 * s - 1.0;
    const double area = g.h[t1] * g.h[t2];
    for (int c = 0; c < 3; ++c) {
      const double nc = c == d ? nd : 0.0;
      for (int p = threadIdx.x; p < N2; p += blockDim.x) {
        const double w = T.gw[p % N] * T.gw[p / N] * area;
        const double nu = nu_face[((size_t)e * 6 + f) * N2 + p];
        const double tau = g.cip * (double)(N * N) * lam * nu;
        double gv[3];
        for (int j = 0; j < 3; ++j) gv[j] = wall_val(wall, g, e, f, p, j, N2);
        CA[p] = -nu * w * (gv[c] * nd + nc * gv[d]) * g.ih[d];
        CB[p] = -nu * w * nc * gv[t1] * g.ih[t1];
        CC[p] = -nu * w * nc * gv[t2] * g.ih[t2];
        CE[p] = 2.0 * tau * w * (gv[c] + nc * gv[d] * nd);
      }
      __syncthreads();
      // normal derivative: every node along the normal line, weight l'_i(s)
      sweep<N, N, 1, 0, N, true>(T.S, N, CA, FT);
      __syncthreads();
      sweep<N, N, 1, 1, N, true>(T.S, N, FT, FR);
      __syncthreads();
      for (int i = threadIdx.x; i < N3; i += blockDim.x) {
        int idx[3] = {i % N, (i / N) % N, i / N2};
        OUT[c][i] += T.dS[s][idx[d]] * FR[idx[t1] + N * idx[t2]];
      }
      __syncthreads();
      // tangential derivatives and values: face nodes only
      sweep<N, N, 1, 0, N, true>(T.DS, N, CB, FT);
      __syncthreads();
      sweep<N, N, 1, 1, N, true>(T.S, N, FT, FR);
      __syncthreads();
      sweep<N, N, 1, 0, N, true>(T.S, N, CC, FT);
      __syncthreads();
      sweep<N, N, 1, 1, N, true>(T.DS, N, FT, CB);
      __syncthreads();
      sweep<N, N, 1, 0, N, true>(T.S, N, CE, FT);
      __syncthreads();
      sweep<N, N, 1, 1, N, true>(T.S, N, FT, CC);
      __syncthreads();
      for (int p = threadIdx.x; p < N2; p += blockDim.x)
        OUT[c][fnode(d, s, p % N, p / N, N)] += FR[p] + CB[p] + CC[p];
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) y[(size_t)e * 3 * N3 + i] = OUT[i / N3][i % N3];
}

// ------------------------------------------------------------------- CFL
template <int N>
__global__ void __launch_bounds__(kSplitThreads) cfl_kernel(LevelGeom g, SplitTab tab, const double* __restrict__ u,
                                                            unsigned long long* __restrict__ vmax_bits) {
  constexpr int N3 = N * N * N;
  __shared__ STabSm T;
  __shared__ double U[3][N3], Q[3][N3], T0[N3], T1[N3];
  __shared__ double red[kSplitThreads];
  const int e = blockIdx.x;
  load_tab(tab, T);
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) U[i / N3][i % N3] = u[(size_t)e * 3 * N3 + i];
  __syncthreads();
  for (int c = 0; c < 3; ++c) sweep3<N, N, false>(T.S, N, U[c], T0, T1, Q[c]);
  double m = 0.0;
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    const double a = Q[0][q] * g.ih[0], b = Q[1][q] * g.ih[1], c = Q[2][q] * g.ih[2];
    m = fmax(m, sqrt(a * a + b * b + c * c));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  // non-negative doubles order like their bit patterns
  if (threadIdx.x == 0) atomicMax(vmax_bits, (unsigned long long)__double_as_longlong(red[0]));
}

// positions of the Gauss points of every boundary face, [nbf][n^2][3]
template <int N>
__global__ void bpoints_kernel(LevelGeom g, SplitTab tab, int nbf, double* __restrict__ xyz) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)nbf * N * N) return;
  const int b = (int)(i / (N * N)), p = (int)(i % (N * N));
  int e, f;
  bface_cell(g, b, &e, &f);
  const int d = f >> 1, s = f & 1;
  int t1, t2;
  face_dirs(d, &t1, &t2);
  int ijk[3];
  cell_ijk(g, e, ijk);
  double xi[3];
  xi[d] = s;
  xi[t1] = tab.gp[p % N];
  xi[t2] = tab.gp[p / N];
  for (int c = 0; c < 3; ++c) xyz[3 * i + c] = g.x0[c] + (ijk[c] + xi[c]) * g.h[c];
}

}  // namespace

Wall make_wall(const WallArg& a) {
  Wall w{};
  for (int i = 0; i < 18; ++i) w.g[i / 3][i % 3] = a.side ? a.side[i] : 0.0;
  w.pts = a.pts;
  return w;
}

#define SIPG_SPLIT_DISPATCH(NN, CALL) \
  switch (NN) {                       \
    case 3: { constexpr int N = 3; CALL; break; } \
    case 4: { constexpr int N = 4; CALL; break; } \
    case 5: { constexpr int N = 5; CALL; break; } \
    case 6: { constexpr int N = 6; CALL; break; } \
    default: return cudaErrorInvalidValue;        \
  }

cudaError_t launch_convective(int n, const LevelGeom& g, const SplitTab& tab, const WallArg& wall_g,
                              const double* u, double* y, cudaStream_t st) {
  const Wall w = make_wall(wall_g);
  if (g.ncells == 0) return cudaSuccess;
  SIPG_SPLIT_DISPATCH(n, (conv_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, w, u, y)));
  return cudaGetLastError();
}

cudaError_t launch_convective_lin(int n, const LevelGeom& g, const SplitTab& tab, const WallArg& wall_w,
                                  const WallArg& wall_u, const double* w, const double* u, double* y,
                                  cudaStream_t st) {
  const Wall ww = make_wall(wall_w), wu = make_wall(wall_u);
  if (g.ncells == 0) return cudaSuccess;
  SIPG_SPLIT_DISPATCH(n, (conv_lin_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, ww, wu, w, u, y)));
  return cudaGetLastError();
}

int n_wall_faces(const LevelGeom& g) { return g.nbr ? g.nbf : 2 * (g.ny * g.nz + g.nx * g.nz + g.nx * g.ny); }

cudaError_t launch_ppe_boundary(int n, const LevelGeom& g, const SplitTab& tab, const WallArg& wall_g,
                                const PpeBndArgs& a, const RheologyDev& rh, const double* u0, const double* u1,
                                double* sb, cudaStream_t st) {
  const Wall w = make_wall(wall_g);
  PpeBnd pb{};
  pb.a = a;
  pb.rh = rh;
  const int nbf = n_wall_faces(g);
  if (nbf == 0) return cudaSuccess;
  SIPG_SPLIT_DISPATCH(n, (ppe_bnd_kernel<N><<<nbf, kSplitThreads, 0, st>>>(g, tab, w, pb, u0, u1, sb)));
  return cudaGetLastError();
}

cudaError_t launch_ppe_rhs(int n, const LevelGeom& g, const SplitTab& tab, double coef, const double* uhat,
                           const double* sb, double* r, cudaStream_t st) {
  if (g.ncells == 0) return cudaSuccess;
  SIPG_SPLIT_DISPATCH(n, (ppe_rhs_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, coef, uhat, sb, r)));
  return cudaGetLastError();
}

cudaError_t launch_projection_rhs(int n, const LevelGeom& g, const SplitTab& tab, const double* p, double* y,
                                  cudaStream_t st) {
  if (g.ncells == 0) return cudaSuccess;
  SIPG_SPLIT_DISPATCH(n, (proj_rhs_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, p, y)));
  return cudaGetLastError();
}

cudaError_t launch_viscous_wall_rhs(int n, const LevelGeom& g, const SplitTab& tab, const WallArg& wall_g,
                                    const double* nu_face, double* y, cudaStream_t st) {
  const Wall w = make_wall(wall_g);
  if (g.ncells == 0) return cudaSuccess;
  SIPG_SPLIT_DISPATCH(n, (visc_dir_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, w, nu_face, y)));
  return cudaGetLastError();
}

cudaError_t launch_cfl_max(int n, const LevelGeom& g, const SplitTab& tab, const double* u,
                           unsigned long long* vmax_bits, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(vmax_bits, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess || g.ncells == 0) return e;
  SIPG_SPLIT_DISPATCH(n, (cfl_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, u, vmax_bits)));
  return cudaGetLastError();
}

cudaError_t launch_boundary_points(int n, const LevelGeom& g, const SplitTab& tab, double* xyz, cudaStream_t st) {
  const int nbf = n_wall_faces(g);
  const int64_t total = (int64_t)nbf * n * n;
  if (total == 0) return cudaSuccess;
  const int blocks = (int)((total + 127) / 128);
  SIPG_SPLIT_DISPATCH(n, (bpoints_kernel<N><<<blocks, 128, 0, st>>>(g, tab, nbf, xyz)));
  return cudaGetLastError();
}

}  // namespace sipg
