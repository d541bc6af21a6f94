// Viscosity at the cell and face quadrature points of one level
// (Eq. viscosity_pointwise: nu is precomputed and stored pointwise).
//
// Laws (Sec. 2 and Eq. viscosity_general):
//   constant, analytic nu(x) = 1 + 9 sin^2(pi x) sin^2(pi y) sin^2(pi z),
//   sinker: nu_max inside any sphere |x - c| <= r, nu_matrix outside, then
//           projected element-locally in L2 onto one constant per cell (the
//           raw pointwise indicator gives an indefinite SIPG form),
//   Carreau-Yasuda: eta(gdot) = eta_inf + (eta0 - eta_inf)(kappa + (lambda gdot)^a)^((b-1)/a),
//           gdot = sqrt(2 eps(u):eps(u)), with grad u of the linearization
//           velocity taken on each side from that side's own cell.
// Output: nu_cell [C][n^3] (q = (qz n + qy) n + qx) and nu_face [C][6][n^2]
// (own side, point a + n b over the face's tangential directions t1 < t2).
#include "apply_dispatch.cuh"

namespace sipg {

__device__ __forceinline__ double carreau(const RheologyDev& r, const double G[3][3]) {
  double ee = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const double e = 0.5 * (G[k][l] + G[l][k]);
      ee += e * e;
    }
  const double gdot = sqrt(2.0 * ee);
  return r.eta_inf + (r.eta0 - r.eta_inf) * pow(r.kappa + pow(r.lambda * gdot, r.a), (r.b - 1.0) / r.a);
}

__device__ __forceinline__ double pointwise_nu(const RheologyDev& r, double x, double y, double z) {
  if (r.law == 0) return r.nu;
  if (r.law == 1) {
    const double sx = sin(M_PI * x), sy = sin(M_PI * y), sz = sin(M_PI * z);
    return 1.0 + 9.0 * sx * sx * sy * sy * sz * sz;
  }
  // sinker indicator
  for (int i = 0; i < r.n_spheres; ++i) {
    const double dx = x - r.centers[3 * i], dy = y - r.centers[3 * i + 1], dz = z - r.centers[3 * i + 2];
    if (dx * dx + dy * dy + dz * dz <= r.radius * r.radius) return r.nu_max;
  }
  return r.nu_matrix;
}

// Position-only laws: one thread per (cell, point) of the cell and face rules.
template <int N>
__global__ void viscosity_position_kernel(LevelGeom g, Tab tab, RheologyDev rh, double* nu_cell,
                                          double* nu_face) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const int e = blockIdx.x;
  if (e >= g.ncells) return;
  int ijk[3];
  cell_ijk(g, e, ijk);
  const double o[3] = {g.x0[0] + ijk[0] * g.h[0], g.x0[1] + ijk[1] * g.h[1], g.x0[2] + ijk[2] * g.h[2]};
  __shared__ double part[N3];
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    const int qx = q % N, qy = (q / N) % N, qz = q / N2;
    const double v = pointwise_nu(rh, o[0] + g.h[0] * tab.gp[qx], o[1] + g.h[1] * tab.gp[qy],
                                  o[2] + g.h[2] * tab.gp[qz]);
    nu_cell[(size_t)e * N3 + q] = v;
    part[q] = tab.gw[qx] * tab.gw[qy] * tab.gw[qz] * v;
  }
  if (rh.law == 2) {
    // element-local L2 projection onto a constant (Gauss weights sum to one)
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < N3; ++q) s += part[q];  // fixed order, identical in every thread
    for (int q = threadIdx.x; q < N3; q += blockDim.x) nu_cell[(size_t)e * N3 + q] = s;
    for (int i = threadIdx.x; i < 6 * N2; i += blockDim.x) nu_face[(size_t)e * 6 * N2 + i] = s;
    return;
  }
  for (int i = threadIdx.x; i < 6 * N2; i += blockDim.x) {
    const int f = i / N2, p = i - f * N2;
    const int d = f >> 1, s = f & 1;
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    double xi[3];
    xi[d] = s ? 1.0 : 0.0;
    xi[t1] = tab.gp[p % N];
    xi[t2] = tab.gp[p / N];
    nu_face[(size_t)e * 6 * N2 + i] =
        pointwise_nu(rh, o[0] + g.h[0] * xi[0], o[1] + g.h[1] * xi[1], o[2] + g.h[2] * xi[2]);
  }
}

// Carreau-Yasuda: gradients by sum factorisation (same sweeps as the operator).
template <int N>
__global__ void viscosity_carreau_kernel(LevelGeom g, CTab<double> ct, RheologyDev rh, const double* __restrict__ u,
                                         double* nu_cell, double* nu_face) {
  constexpr int N2 = N * N, N3 = N2 * N;
  __shared__ double dS0[N], dS1[N], gw[N];
  const double* S = ct.S;
  const double* Dg = ct.Dg;
  __shared__ double Xs[3 * N3], U[3 * N3], B1[3 * N3], B2[3 * N3], B3[3 * N3];
  __shared__ double fV[3 * N2], fN[3 * N2], T1[3 * N2], T2[3 * N2], gV[3 * N2], gN[3 * N2],
      gT1[3 * N2], gT2[3 * N2];
  load_tables<N>(ct, dS0, dS1, gw);
  const int e = blockIdx.x;
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) Xs[i] = u[(size_t)e * 3 * N3 + i];
  __syncthreads();
  sweep3<N, 0, false, false>(Xs, B1, S, 3);
  __syncthreads();
  sweep3<N, 1, false, false>(B1, B2, S, 3);
  __syncthreads();
  sweep3<N, 2, false, false>(B2, U, S, 3);
  __syncthreads();
  sweep3<N, 0, false, false>(U, B1, Dg, 3);
  sweep3<N, 1, false, false>(U, B2, Dg, 3);
  sweep3<N, 2, false, false>(U, B3, Dg, 3);
  __syncthreads();
  const double ih[3] = {g.ih[0], g.ih[1], g.ih[2]};
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    double G[3][3];
    const double* Bl[3] = {B1, B2, B3};
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) G[k][l] = Bl[l][k * N3 + q] * ih[l];
    nu_cell[(size_t)e * N3 + q] = carreau(rh, G);
  }
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    const int layer = s ? N - 1 : 0;
    const double* dS = s ? dS1 : dS0;
    const int std_ = dir_stride<N>(d);
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * N2; i += blockDim.x) {
      const int t = i / N2, p = i - t * N2;
      const double* xs = Xs + t * N3 + face_node<N>(d, 0, p % N, p / N);
      double dn = 0.0;
      for (int j = 0; j < N; ++j) dn += dS[j] * xs[j * std_];
      fV[i] = xs[layer * std_];
      fN[i] = dn;
    }
    __syncthreads();
    sweep2<N, 0, false, false>(fV, T1, S, 3);
    sweep2<N, 0, false, false>(fN, T2, S, 3);
    __syncthreads();
    sweep2<N, 1, false, false>(T1, gV, S, 3);
    sweep2<N, 1, false, false>(T2, gN, S, 3);
    __syncthreads();
    sweep2<N, 0, false, false>(gV, gT1, Dg, 3);
    sweep2<N, 1, false, false>(gV, gT2, Dg, 3);
    __syncthreads();
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      double G[3][3];
      for (int k = 0; k < 3; ++k) {
        G[k][d] = gN[k * N2 + p] * ih[d];
        G[k][t1] = gT1[k * N2 + p] * ih[t1];
        G[k][t2] = gT2[k * N2 + p] * ih[t2];
      }
      nu_face[((size_t)e * 6 + f) * N2 + p] = carreau(rh, G);
    }
  }
}

template <int N>
cudaError_t launch_viscosity_n(const LevelGeom& g, const Tab& tab, const RheologyDev& rh, const double* u,
                               double* nu_cell, double* nu_face, cudaStream_t st) {
  if (g.ncells == 0) return cudaSuccess;
  if (rh.law == 3)
    viscosity_carreau_kernel<N><<<g.ncells, 64, 0, st>>>(g, make_ctab<double>(tab), rh, u, nu_cell, nu_face);
  else
    viscosity_position_kernel<N><<<g.ncells, 64, 0, st>>>(g, tab, rh, nu_cell, nu_face);
  return cudaGetLastError();
}

cudaError_t launch_viscosity(int n, const LevelGeom& g, const Tab& tab, const RheologyDev& rh,
                             const double* u, double* nu_cell, double* nu_face, cudaStream_t st) {
  switch (n) {
    case 2: return launch_viscosity_n<2>(g, tab, rh, u, nu_cell, nu_face, st);
    case 3: return launch_viscosity_n<3>(g, tab, rh, u, nu_cell, nu_face, st);
    case 4: return launch_viscosity_n<4>(g, tab, rh, u, nu_cell, nu_face, st);
    case 5: return launch_viscosity_n<5>(g, tab, rh, u, nu_cell, nu_face, st);
    case 6: return launch_viscosity_n<6>(g, tab, rh, u, nu_cell, nu_face, st);
    default: return cudaErrorInvalidValue;
  }
}

// Physical coordinates of the Gauss-Lobatto nodes, [C][n^3][3].
template <int N>
__global__ void node_points_kernel(LevelGeom g, Tab tab, double* xyz) {
  constexpr int N3 = N * N * N;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)g.ncells * N3) return;
  const int e = (int)(i / N3), r = (int)(i % N3);
  int ijk[3];
  cell_ijk(g, e, ijk);
  xyz[3 * i + 0] = g.x0[0] + (ijk[0] + tab.gll[r % N]) * g.h[0];
  xyz[3 * i + 1] = g.x0[1] + (ijk[1] + tab.gll[(r / N) % N]) * g.h[1];
  xyz[3 * i + 2] = g.x0[2] + (ijk[2] + tab.gll[r / (N * N)]) * g.h[2];
}

cudaError_t launch_node_points(int n, const LevelGeom& g, const Tab& tab, double* xyz, cudaStream_t st) {
  const int64_t total = (int64_t)g.ncells * n * n * n;
  const int blocks = (int)((total + 255) / 256);
  if (blocks == 0) return cudaSuccess;
  switch (n) {
    case 2: node_points_kernel<2><<<blocks, 256, 0, st>>>(g, tab, xyz); break;
    case 3: node_points_kernel<3><<<blocks, 256, 0, st>>>(g, tab, xyz); break;
    case 4: node_points_kernel<4><<<blocks, 256, 0, st>>>(g, tab, xyz); break;
    case 5: node_points_kernel<5><<<blocks, 256, 0, st>>>(g, tab, xyz); break;
    case 6: node_points_kernel<6><<<blocks, 256, 0, st>>>(g, tab, xyz); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace sipg

namespace sipg {

// Cellwise-constant viscosity carried to the next coarser level: the same
// value on a p-level (same cells), the mean of the 8 children on an h-level
// (the L2 projection of the piecewise constant). Written to every cell and
// face point of the coarse cell.
__global__ void cell_nu_transfer_kernel(LevelGeom fine, LevelGeom coarse, int kind, int nf3, int nc3, int nc2,
                                        const double* __restrict__ fine_cell, double* __restrict__ nu_cell,
                                        double* __restrict__ nu_face) {
  const int ec = blockIdx.x;
  if (ec >= coarse.ncells) return;
  double v;
  if (kind == 1) {
    v = fine_cell[(size_t)ec * nf3];
  } else {
    int ci[3];
    cell_ijk(coarse, ec, ci);
    v = 0.0;
    for (int ch = 0; ch < 8; ++ch) {
      const int ef = grid_cell(fine, 2 * ci[0] + (ch & 1), 2 * ci[1] + ((ch >> 1) & 1), 2 * ci[2] + (ch >> 2));
      v += fine_cell[(size_t)ef * nf3];
    }
    v *= 0.125;
  }
  for (int i = threadIdx.x; i < nc3; i += blockDim.x) nu_cell[(size_t)ec * nc3 + i] = v;
  for (int i = threadIdx.x; i < 6 * nc2; i += blockDim.x) nu_face[(size_t)ec * 6 * nc2 + i] = v;
}

cudaError_t launch_cell_nu_transfer(const LevelGeom& fine, const LevelGeom& coarse, int kind, int nf, int nc,
                                    const double* fine_cell, double* nu_cell, double* nu_face, cudaStream_t st) {
  if (coarse.ncells == 0) return cudaSuccess;
  cell_nu_transfer_kernel<<<coarse.ncells, 64, 0, st>>>(fine, coarse, kind, nf * nf * nf, nc * nc * nc, nc * nc,
                                                       fine_cell, nu_cell, nu_face);
  return cudaGetLastError();
}

}  // namespace sipg
