// SIPG viscous and Poisson operators on trilinear (non-affine) hexahedra,
// Sec. 5 of the paper on general hexahedral cells (the jittered channel mesh
// of the backward-facing-step workload). Same forms, fluxes, mirror boundary
// conditions and penalty as the affine kernels (operator.cuh); the geometry is
// evaluated per quadrature point from the cell's 8 vertices:
//   J = dx/dxi of the trilinear map, W = w det J, grad = J^-T grad_xi;
//   faces: n = +-(t1 x t2)/|t1 x t2| from the tangents t = dx/dxi_t, surface
//   weight w_a w_b |t1 x t2|; Lambda_e = sum_f w_f |f| / |Omega_e| from the
//   integrated areas and volume (mapped_lambda_kernel).
// The topology is structured (cells (i, j, k), neighbours across the faces),
// vertex (i, j, k) at verts[((k (ny+1) + j)(nx+1) + i) * 3 + c].
//
// The operator kernels read the geometry of every quadrature point from
// per-level metric arrays built once per mesh (mapped_metric_kernel, FP64 with
// an FP32 copy), the scheme of matrix-free codes on general cells:
//   cell point q:      J^-1 (9 entries), W = w_q det J             [cell][10][n^3]
//   face f, point p:   J^-1 of the own side (9), the unit normal n (3, outward
//                      of the own cell), W = w_a w_b |t1 x t2|      [cell][6][13][n^2]
// and the neighbour's J^-1 at the same face point from the neighbour's entry of
// its opposite face (same tangential coordinates on the structured grid).
// Without them every point re-evaluated the trilinear Jacobian from the 8
// vertices (about 100 flops per point, twice per face point), which made the
// FP64 apply twice as expensive as the affine one and the FP32 applies
// latency bound. The other trilinear forms (mass, diagonal, step forms) still
// evaluate the geometry from the vertices: they run once per setup or step.
#include "kernels.cuh"
#include "mapped_geom.cuh"
#include "sweeps.cuh"

// Cells per CTA of the trilinear apply: at low degree one cell
// leaves most lanes idle between the barriers of its sweeps (n^3 = 8 or 27
// points), so several cells share a CTA and every phase runs over all of them;
// the tensors live in dynamic shared memory. Measured at 32^3, 5 % jitter (FP32
// level applies k = 3 / 2 / 1 viscous and k = 2 pressure, ms): 2 / 4 / 8 cells
// 1.17 / 0.58 / 0.24 / 0.36, twice that 0.84 / 0.52 / 0.16 / 0.27, three times
// 0.82 / 0.49 / 0.14 / 0.22, four times 0.93 / 0.71 / 0.14 / 0.29; the FP64
// apply (bound by the FP64 pipe) is slower with more cells (3.88 -> 4.44 ms).
// Resident CTAs per SM requested from the compiler: one cell per CTA measured at
// 32^3, k = 3: 2 CTAs 22.5 ms, 4 (128 registers) 12.7 ms, 8 (64 registers)
// 11.1 ms; with the stored metric the budget of 4 keeps every instance unspilled.
template <int N, typename R = double> struct MappedCfg {
  static constexpr int CB = (N == 2 ? 8 : (N == 3 ? 4 : (N == 4 ? 2 : 1))) * (sizeof(R) == 4 && N <= 4 ? 3 : 1);
};
// Threads per CTA and resident CTAs requested from the compiler: the FP32
// instances are latency bound at 12 resident warps per SM (three 4-warp CTAs by
// shared memory); measured FP32 level applies at 32^3 (ms, 128 / 192 / 256
// threads): n = 4 viscous 0.83 / 0.80 / 0.78, n = 3 viscous 0.39 / 0.37 / 0.41,
// n = 3 pressure 0.21 / 0.24 / 0.25, n = 2 viscous 0.14 / 0.16 / 0.16.
template <int N, int NC, typename R> struct MappedLaunch {
  static constexpr bool F32 = sizeof(R) == 4;
  static constexpr int THREADS = F32 && N == 4 ? 256 : (F32 && N == 3 && NC == 3 ? 192 : sipg::sweeps::kSplitThreads);
  static constexpr int MIN_BLOCKS = THREADS > sipg::sweeps::kSplitThreads ? 3 : (N <= 4 ? 4 : (N == 5 ? 6 : 4));
};
// dynamic shared memory of the apply (elements of R): U, Q, G[3], T0, T1, OUT
// (n^3 per tensor) and FM, FP, CF (4 n^2), SC (8 n^2) per tensor of the CTA
template <int N, int NC, typename R>
constexpr size_t mapped_apply_smem() {
  return sizeof(R) * (size_t)MappedCfg<N, R>::CB * NC * (8 * N * N * N + 20 * N * N);
}

namespace sipg {
namespace {
using namespace sweeps;
using namespace mgeo;
// Metric terms of one level (see the header): one CTA per cell, FP64, stored in
// FP64 and rounded to FP32.
template <int N>
__global__ void __launch_bounds__(kSplitThreads) mapped_metric_kernel(LevelGeom g, SplitTab tab,
                                                                      const double* __restrict__ verts,
                                                                      double* __restrict__ cmet64,
                                                                      float* __restrict__ cmet32,
                                                                      double* __restrict__ fmet64,
                                                                      float* __restrict__ fmet32) {
  constexpr int N3 = N * N * N, N2 = N * N;
  __shared__ double X[8][3];
  const int e = blockIdx.x;
  load_cell_vertices(g, verts, e, X);
  __syncthreads();
  const size_t cb = (size_t)e * 10 * N3;
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    const int qx = q % N, qy = (q / N) % N, qz = q / N2;
    double J[3][3], Ji[3][3];
    trilinear_jac<double>(X, tab.gp[qx], tab.gp[qy], tab.gp[qz], J);
    const double det = inverse3(J, Ji);
    double v[10];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) v[3 * a + b] = Ji[a][b];
    v[9] = tab.gw[qx] * tab.gw[qy] * tab.gw[qz] * det;
    for (int k = 0; k < 10; ++k) {
      cmet64[cb + (size_t)k * N3 + q] = v[k];
      cmet32[cb + (size_t)k * N3 + q] = (float)v[k];
    }
  }
  for (int i = threadIdx.x; i < 6 * N2; i += blockDim.x) {
    const int f = i / N2, p = i - f * N2;
    const int d = f >> 1, s = f & 1;
    int t1, t2;
    face_dirs(d, &t1, &t2);
    double xi[3];
    xi[d] = s ? 1.0 : 0.0;
    xi[t1] = tab.gp[p % N];
    xi[t2] = tab.gp[p / N];
    double J[3][3], Ji[3][3];
    trilinear_jac<double>(X, xi[0], xi[1], xi[2], J);
    inverse3(J, Ji);
    const double ta[3] = {J[0][t1], J[1][t1], J[2][t1]}, tb[3] = {J[0][t2], J[1][t2], J[2][t2]};
    double n[3] = {ta[1] * tb[2] - ta[2] * tb[1], ta[2] * tb[0] - ta[0] * tb[2], ta[0] * tb[1] - ta[1] * tb[0]};
    const double area = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    const double orient = (2.0 * s - 1.0) * (d == 1 ? -1.0 : 1.0);
    double v[13];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) v[3 * a + b] = Ji[a][b];
    for (int k = 0; k < 3; ++k) v[9 + k] = n[k] * (orient / area);
    v[12] = tab.gw[p % N] * tab.gw[p / N] * area;
    const size_t fb = ((size_t)e * 6 + f) * 13 * N2;
    for (int k = 0; k < 13; ++k) {
      fmet64[fb + (size_t)k * N2 + p] = v[k];
      fmet32[fb + (size_t)k * N2 + p] = (float)v[k];
    }
  }
}

template <int N, int NC, typename R>
__global__ void __launch_bounds__(MappedLaunch<N, NC, R>::THREADS, MappedLaunch<N, NC, R>::MIN_BLOCKS) mapped_apply_kernel(LevelGeom g, SplitTab tab,
                                                                     mgeo::MTab<R> mt,
                                                                     const R* __restrict__ cmet,
                                                                     const R* __restrict__ fmet,
                                                                     const double* __restrict__ lam,
                                                                     const R* __restrict__ nu_cell,
                                                                     const R* __restrict__ nu_face, double mass_d,
                                                                     const R* __restrict__ x,
                                                                     R* __restrict__ y, int64_t batch_stride) {
  constexpr int N3 = N * N * N, N2 = N * N, CB = MappedCfg<N, R>::CB, NT = CB * NC;
  __shared__ STabSmT<R> T;
  __shared__ int NB[CB];
  extern __shared__ __align__(16) unsigned char msm_raw[];
  R* msm = reinterpret_cast<R*>(msm_raw);
  R(*U)[N3] = reinterpret_cast<R(*)[N3]>(msm);
  R(*Q)[N3] = reinterpret_cast<R(*)[N3]>(msm + 1 * NT * N3);
  R(*G)[NT][N3] = reinterpret_cast<R(*)[NT][N3]>(msm + 2 * NT * N3);
  R(*T0)[N3] = reinterpret_cast<R(*)[N3]>(msm + 5 * NT * N3);
  R(*T1)[N3] = reinterpret_cast<R(*)[N3]>(msm + 6 * NT * N3);
  R(*OUT)[N3] = reinterpret_cast<R(*)[N3]>(msm + 7 * NT * N3);
  R* fbase = msm + 8 * NT * N3;
  R(*FM)[4 * N2] = reinterpret_cast<R(*)[4 * N2]>(fbase);
  R(*FP)[4 * N2] = reinterpret_cast<R(*)[4 * N2]>(fbase + 4 * NT * N2);
  R(*CF)[4 * N2] = reinterpret_cast<R(*)[4 * N2]>(fbase + 8 * NT * N2);
  R* SC = fbase + 12 * NT * N2;
  const R mass = (R)mass_d;
  x += (int64_t)blockIdx.y * batch_stride;
  y += (int64_t)blockIdx.y * batch_stride;
  const int e0 = blockIdx.x * CB, last = g.ncells - 1;
  load_tab(tab, T);
  for (int i = threadIdx.x; i < NT * N3; i += blockDim.x) {
    const int b = i / N3, c = b / NC;
    U[b][i - b * N3] = x[(size_t)min(e0 + c, last) * NC * N3 + (b - c * NC) * N3 + (i - b * N3)];
  }
  __syncthreads();
  // ---- cell term
  if constexpr (mapped_line_sweeps<N>()) {
    lsweep<N, 0, false, false>(mt.S, U[0], T0[0], NT);
    __syncthreads();
    lsweep<N, 1, false, false>(mt.S, T0[0], T1[0], NT);
    __syncthreads();
    lsweep<N, 2, false, false>(mt.S, T1[0], Q[0], NT);
    __syncthreads();
    lsweep<N, 0, false, false>(mt.Dg, Q[0], G[0][0], NT);
    lsweep<N, 1, false, false>(mt.Dg, Q[0], G[1][0], NT);
    lsweep<N, 2, false, false>(mt.Dg, Q[0], G[2][0], NT);
  } else {
    sweep3b<N, N, false>(T.S, N, U[0], T0[0], T1[0], Q[0], NT);
    for (int m = 0; m < 3; ++m) sweep_dirb<N, false>(m, T.Dg, Q[0], G[m][0], NT);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < CB * N3; i += blockDim.x) {
    const int c = i / N3, q = i - c * N3;
    const int e = min(e0 + c, last);
    const R* cm = cmet + (size_t)e * 10 * N3 + q;
    R Ji[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Ji[a][b] = cm[(3 * a + b) * N3];
    const R W = cm[9 * N3];
    R Gp[NC][3];
    for (int k = 0; k < NC; ++k) {
      const int b = c * NC + k;
      for (int l = 0; l < 3; ++l) Gp[k][l] = G[0][b][q] * Ji[0][l] + G[1][b][q] * Ji[1][l] + G[2][b][q] * Ji[2][l];
    }
    R Tf[NC][3];
    if (NC == 3) {
      const R nu = nu_cell[(size_t)e * N3 + q];
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) Tf[k][l] = nu * (Gp[k][l] + Gp[l][k]);  // 2 nu eps(u)
    } else {
      for (int l = 0; l < 3; ++l) Tf[0][l] = Gp[0][l];
    }
    for (int k = 0; k < NC; ++k) {
      const int b = c * NC + k;
      for (int m = 0; m < 3; ++m) G[m][b][q] = W * (Tf[k][0] * Ji[m][0] + Tf[k][1] * Ji[m][1] + Tf[k][2] * Ji[m][2]);
      Q[b][q] = mass * W * Q[b][q];
    }
  }
  __syncthreads();
  // Q += Dx^T Gx + Dy^T Gy + Dz^T Gz, then S^T along x, y, z
  if constexpr (mapped_line_sweeps<N>()) {
    lsweep<N, 0, true, true>(mt.Dg, G[0][0], Q[0], NT);
    __syncthreads();
    lsweep<N, 1, true, true>(mt.Dg, G[1][0], Q[0], NT);
    __syncthreads();
    lsweep<N, 2, true, true>(mt.Dg, G[2][0], Q[0], NT);
    __syncthreads();
    lsweep<N, 0, true, false>(mt.S, Q[0], T0[0], NT);
    __syncthreads();
    lsweep<N, 1, true, false>(mt.S, T0[0], T1[0], NT);
    __syncthreads();
    lsweep<N, 2, true, false>(mt.S, T1[0], OUT[0], NT);
    __syncthreads();
  } else {
    for (int m = 0; m < 3; ++m) {
      sweep_dirb<N, true>(m, T.Dg, G[m][0], T0[0], NT);
      __syncthreads();
      for (int i = threadIdx.x; i < NT * N3; i += blockDim.x) Q[0][i] += T0[0][i];
      __syncthreads();
    }
    sweep3b<N, N, true>(T.S, N, Q[0], T0[0], T1[0], OUT[0], NT);
  }
  // ---- faces
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    int t1, t2;
    face_dirs(d, &t1, &t2);
    const int fo = 2 * d + (1 - s);
    for (int c = threadIdx.x; c < CB; c += blockDim.x) NB[c] = cell_neighbor(g, min(e0 + c, last), f);
    __syncthreads();
    face_evalb<N>([&](int b, int i) { return U[b][i]; }, d, s, T, mt, FM[0], SC, NT);
    face_evalb<N>(
        [&](int b, int i) {
          const int nb = NB[b / NC];
          return nb >= 0 ? x[(size_t)nb * NC * N3 + (b % NC) * N3 + i] : R(0);
        },
        d, 1 - s, T, mt, FP[0], SC, NT);
    for (int i = threadIdx.x; i < CB * N2; i += blockDim.x) {
      const int c = i / N2, p = i - c * N2;
      const int e = min(e0 + c, last);
      const int nb = NB[c];
      const bool neumann = nb < 0 && face_bc(g, e, f) == 1;  // homogeneous Neumann: no term
      const R lam_e = (R)lam[e];
      const R lam_p = nb >= 0 ? (R)lam[nb] : lam_e;
      const R tau0 = R(g.cip * (double)(N * N)) * (lam_e > lam_p ? lam_e : lam_p);
      const R* fm = fmet + ((size_t)e * 6 + f) * 13 * N2 + p;
      const R* fq = fmet + ((size_t)(nb >= 0 ? nb : e) * 6 + (nb >= 0 ? fo : f)) * 13 * N2 + p;
      R Jim[3][3], Jip[3][3], n[3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          Jim[a][b] = fm[(3 * a + b) * N2];
          Jip[a][b] = fq[(3 * a + b) * N2];
        }
#pragma unroll
      for (int k = 0; k < 3; ++k) n[k] = fm[(9 + k) * N2];
      const R W = fm[12 * N2];
      // physical traces
      R um[NC], up[NC], Gm[NC][3], Gq[NC][3];
      for (int k = 0; k < NC; ++k) {
        const R* fm = FM[c * NC + k];
        const R* fp = FP[c * NC + k];
        R rm[3], rp[3];
        rm[d] = fm[N2 + p];
        rm[t1] = fm[2 * N2 + p];
        rm[t2] = fm[3 * N2 + p];
        um[k] = fm[p];
        for (int l = 0; l < 3; ++l) Gm[k][l] = rm[0] * Jim[0][l] + rm[1] * Jim[1][l] + rm[2] * Jim[2][l];
        if (nb >= 0) {
          rp[d] = fp[N2 + p];
          rp[t1] = fp[2 * N2 + p];
          rp[t2] = fp[3 * N2 + p];
          up[k] = fp[p];
          for (int l = 0; l < 3; ++l) Gq[k][l] = rp[0] * Jip[0][l] + rp[1] * Jip[1][l] + rp[2] * Jip[2][l];
        } else {  // Dirichlet mirror
          up[k] = -um[k];
          for (int l = 0; l < 3; ++l) Gq[k][l] = Gm[k][l];
        }
      }
      R cv[NC], S[NC][3];
      if (NC == 3) {
        const R num = nu_face[((size_t)e * 6 + f) * N2 + p];
        const R nup = nb >= 0 ? nu_face[((size_t)nb * 6 + fo) * N2 + p] : num;
        R nub = num > nup ? num : nup;
        if (g.face_nu == 1) nub = R(0.5) * (num + nup);
        if (g.face_nu == 2) nub = R(2) * num * nup / (num + nup);
        const R tau = tau0 * nub;
        R jm[3], jn = R(0);
        for (int k = 0; k < 3; ++k) {
          jm[k] = um[k] - up[k];
          jn += jm[k] * n[k];
        }
        for (int k = 0; k < 3; ++k) {
          // (A + A^T) n, A = (nu- Gm + nu+ Gp)/2
          R an = R(0);
          for (int l = 0; l < 3; ++l)
            an += R(0.5) * (num * (Gm[k][l] + Gm[l][k]) + nup * (Gq[k][l] + Gq[l][k])) * n[l];
          cv[k] = W * (-an + tau * (jm[k] + n[k] * jn));
          for (int l = 0; l < 3; ++l) S[k][l] = -W * num * R(0.5) * (jm[k] * n[l] + jm[l] * n[k]);
        }
      } else {
        const R tau = tau0;
        const R jm = um[0] - up[0];
        R gn = R(0);
        for (int l = 0; l < 3; ++l) gn += R(0.5) * (Gm[0][l] + Gq[0][l]) * n[l];
        cv[0] = W * (-gn + tau * jm);
        for (int l = 0; l < 3; ++l) S[0][l] = -W * R(0.5) * jm * n[l];
      }
      for (int k = 0; k < NC; ++k) {
        R* cf = CF[c * NC + k];
        R Rv[3];
        for (int m = 0; m < 3; ++m) Rv[m] = S[k][0] * Jim[m][0] + S[k][1] * Jim[m][1] + S[k][2] * Jim[m][2];
        cf[p] = neumann ? R(0) : cv[k];
        cf[N2 + p] = neumann ? R(0) : Rv[d];
        cf[2 * N2 + p] = neumann ? R(0) : Rv[t1];
        cf[3 * N2 + p] = neumann ? R(0) : Rv[t2];
      }
    }
    __syncthreads();
    face_eval_tb<N>(CF[0], d, s, T, mt, OUT[0], SC, NT);
  }
  for (int i = threadIdx.x; i < NT * N3; i += blockDim.x) {
    const int c = (i / N3) / NC;
    if (e0 + c <= last) y[(size_t)e0 * NC * N3 + i] = OUT[0][i];
  }
}

// Lambda_e = sum_f w_f |f| / |Omega_e| (w = 1/2 interior, 1 boundary), one thread per cell
__global__ void mapped_lambda_kernel(LevelGeom g, SplitTab tab, int n, const double* __restrict__ verts,
                                     double* __restrict__ lam) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.ncells) return;
  double X[8][3];
  int ijk[3];
  cell_ijk(g, e, ijk);
  const int i = ijk[0], j = ijk[1], k = ijk[2];
  for (int v = 0; v < 8; ++v) {
    const int a = v & 1, b = (v >> 1) & 1, c = (v >> 2) & 1;
    const size_t idx = ((size_t)(k + c) * (g.ny + 1) + (j + b)) * (g.nx + 1) + (i + a);
    for (int t = 0; t < 3; ++t) X[v][t] = verts[idx * 3 + t];
  }
  double vol = 0.0, J[3][3], Ji[3][3];
  for (int q = 0; q < n * n * n; ++q) {
    const int qx = q % n, qy = (q / n) % n, qz = q / (n * n);
    trilinear_jac(X, tab.gp[qx], tab.gp[qy], tab.gp[qz], J);
    vol += tab.gw[qx] * tab.gw[qy] * tab.gw[qz] * inverse3(J, Ji);
  }
  double acc = 0.0;
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    double area = 0.0;
    for (int p = 0; p < n * n; ++p) {
      double xi[3];
      xi[d] = s ? 1.0 : 0.0;
      xi[t1] = tab.gp[p % n];
      xi[t2] = tab.gp[p / n];
      trilinear_jac(X, xi[0], xi[1], xi[2], J);
      const double c0 = J[1][t1] * J[2][t2] - J[2][t1] * J[1][t2];
      const double c1 = J[2][t1] * J[0][t2] - J[0][t1] * J[2][t2];
      const double c2 = J[0][t1] * J[1][t2] - J[1][t1] * J[0][t2];
      area += tab.gw[p % n] * tab.gw[p / n] * sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    }
    acc += (cell_neighbor(g, e, f) >= 0 ? 0.5 : 1.0) * area;
  }
  lam[e] = acc / vol;
}

// nu at the cell and face Gauss points of trilinear cells (Eq. viscosity_pointwise):
// law 0 constant, 1 analytic (position), 2 sphere field (position, then the
// element-local projection onto a constant with the weights w det J),
// 3 Carreau-Yasuda (physical gradient of u)
template <int N>
__global__ void __launch_bounds__(kSplitThreads) mapped_viscosity_kernel(LevelGeom g, SplitTab tab,
                                                                         const double* __restrict__ verts,
                                                                         RheologyDev rh,
                                                                         const double* __restrict__ u,
                                                                         double* __restrict__ nu_cell,
                                                                         double* __restrict__ nu_face) {
  constexpr int N3 = N * N * N, N2 = N * N;
  __shared__ STabSm T;
  __shared__ double X[8][3];
  __shared__ double U[3][N3], Q[3][N3], G[3][3][N3], T0[N3], T1[N3];
  __shared__ double FM[3][4 * N2], SC[5 * N2], red[2][kSplitThreads];
  const int e = blockIdx.x;
  load_tab(tab, T);
  load_cell_vertices(g, verts, e, X);
  const bool carreau = rh.law == 3;
  if (carreau)
    for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) U[i / N3][i % N3] = u[(size_t)e * 3 * N3 + i];
  __syncthreads();
  if (carreau) {
    for (int c = 0; c < 3; ++c) sweep3<N, N, false>(T.S, N, U[c], T0, T1, Q[c]);
    for (int c = 0; c < 3; ++c)
      for (int m = 0; m < 3; ++m) sweep_dir<N, false>(m, T.Dg, Q[c], G[c][m]);
    __syncthreads();
  }
  auto point_nu = [&](const double pos[3], const double Gp[3][3]) -> double {
    if (rh.law == 0) return rh.nu;
    if (rh.law == 1) {
      const double sx = sin(M_PI * pos[0]), sy = sin(M_PI * pos[1]), sz = sin(M_PI * pos[2]);
      return 1.0 + 9.0 * sx * sx * sy * sy * sz * sz;
    }
    if (rh.law == 2) {
      for (int i = 0; i < rh.n_spheres; ++i) {
        const double dx = pos[0] - rh.centers[3 * i], dy = pos[1] - rh.centers[3 * i + 1],
                     dz = pos[2] - rh.centers[3 * i + 2];
        if (dx * dx + dy * dy + dz * dz <= rh.radius * rh.radius) return rh.nu_max;
      }
      return rh.nu_matrix;
    }
    double ee = 0.0;
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) {
        const double v = 0.5 * (Gp[k][l] + Gp[l][k]);
        ee += v * v;
      }
    const double gdot = sqrt(2.0 * ee);
    return rh.eta_inf + (rh.eta0 - rh.eta_inf) * pow(rh.kappa + pow(rh.lambda * gdot, rh.a), (rh.b - 1.0) / rh.a);
  };
  double wsum = 0.0, nsum = 0.0;
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    const int qx = q % N, qy = (q / N) % N, qz = q / N2;
    double J[3][3], Ji[3][3], pos[3], Gp[3][3] = {{0}};
    trilinear_jac(X, tab.gp[qx], tab.gp[qy], tab.gp[qz], J, pos);
    const double det = inverse3(J, Ji);
    if (carreau)
      for (int c = 0; c < 3; ++c)
        for (int l = 0; l < 3; ++l) Gp[c][l] = G[c][0][q] * Ji[0][l] + G[c][1][q] * Ji[1][l] + G[c][2][q] * Ji[2][l];
    const double nu = point_nu(pos, Gp);
    nu_cell[(size_t)e * N3 + q] = nu;
    const double w = T.gw[qx] * T.gw[qy] * T.gw[qz] * det;
    wsum += w;
    nsum += w * nu;
  }
  if (rh.law == 2) {  // sphere field: element-local L2 projection onto a constant
    red[0][threadIdx.x] = wsum;
    red[1][threadIdx.x] = nsum;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        red[0][threadIdx.x] += red[0][threadIdx.x + w];
        red[1][threadIdx.x] += red[1][threadIdx.x + w];
      }
      __syncthreads();
    }
    const double nu_e = red[1][0] / red[0][0];
    for (int q = threadIdx.x; q < N3; q += blockDim.x) nu_cell[(size_t)e * N3 + q] = nu_e;
    for (int p = threadIdx.x; p < 6 * N2; p += blockDim.x) nu_face[(size_t)e * 6 * N2 + p] = nu_e;
    return;
  }
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    int t1, t2;
    face_dirs(d, &t1, &t2);
    if (carreau)
      for (int c = 0; c < 3; ++c) face_eval<N>(U[c], d, s, T, FM[c], SC);
    __syncthreads();
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      double xi[3];
      xi[d] = s ? 1.0 : 0.0;
      xi[t1] = tab.gp[p % N];
      xi[t2] = tab.gp[p / N];
      double J[3][3], Ji[3][3], pos[3], Gp[3][3] = {{0}};
      trilinear_jac(X, xi[0], xi[1], xi[2], J, pos);
      inverse3(J, Ji);
      if (carreau)
        for (int c = 0; c < 3; ++c) {
          double r[3];
          r[d] = FM[c][N2 + p];
          r[t1] = FM[c][2 * N2 + p];
          r[t2] = FM[c][3 * N2 + p];
          for (int l = 0; l < 3; ++l) Gp[c][l] = r[0] * Ji[0][l] + r[1] * Ji[1][l] + r[2] * Ji[2][l];
        }
      nu_face[((size_t)e * 6 + f) * N2 + p] = point_nu(pos, Gp);
    }
    __syncthreads();
  }
}

}  // namespace

#define SIPG_MAPPED_DISPATCH(NN, CALL)              \
  switch (NN) {                                     \
    case 2: { constexpr int N = 2; CALL; break; }   \
    case 3: { constexpr int N = 3; CALL; break; }   \
    case 4: { constexpr int N = 4; CALL; break; }   \
    case 5: { constexpr int N = 5; CALL; break; }   \
    case 6: { constexpr int N = 6; CALL; break; }   \
    default: return cudaErrorInvalidValue;          \
  }

cudaError_t launch_mapped_metric(int n, const LevelGeom& g, const SplitTab& tab, const double* verts, double* cmet64,
                                 float* cmet32, double* fmet64, float* fmet32, cudaStream_t st) {
  if (g.ncells == 0) return cudaSuccess;
  SIPG_MAPPED_DISPATCH(n, (mapped_metric_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, verts, cmet64, cmet32,
                                                                                       fmet64, fmet32)));
  return cudaGetLastError();
}

// one launch of the trilinear apply: shared-memory opt-in once per instantiation
template <int N, int NC, typename R>
cudaError_t launch_mapped_apply_n(const LevelGeom& g, const SplitTab& tab, const R* cmet, const R* fmet,
                                  const double* lam, const R* nu_cell, const R* nu_face, double mass, const R* x, R* y,
                                  int nbatch, cudaStream_t st) {
  constexpr size_t smem = mapped_apply_smem<N, NC, R>();
  static bool attr_set = false;  // per instantiation, per process (single device)
  if (!attr_set) {
    const cudaError_t e =
        cudaFuncSetAttribute(mapped_apply_kernel<N, NC, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  constexpr int cb = MappedCfg<N, R>::CB;
  const int64_t stride = (int64_t)g.ncells * NC * N * N * N;
  const dim3 grid((g.ncells + cb - 1) / cb, nbatch);
  mapped_apply_kernel<N, NC, R><<<grid, MappedLaunch<N, NC, R>::THREADS, smem, st>>>(g, tab, mgeo::make_mtab<R>(tab), cmet, fmet, lam,
                                                                     nu_cell, nu_face, mass, x, y, stride);
  return cudaGetLastError();
}

cudaError_t launch_mapped_apply(int n, int ncomp, const LevelGeom& g, const SplitTab& tab, const double* cmet,
                                const double* fmet, const double* lam, const double* nu_cell, const double* nu_face,
                                double mass, const double* x, double* y, int nbatch, cudaStream_t st) {
  if (g.ncells == 0 || nbatch == 0) return cudaSuccess;
  if (ncomp == 3) {
    SIPG_MAPPED_DISPATCH(n, return (launch_mapped_apply_n<N, 3, double>(g, tab, cmet, fmet, lam, nu_cell, nu_face,
                                                                        mass, x, y, nbatch, st)));
  } else {
    SIPG_MAPPED_DISPATCH(n, return (launch_mapped_apply_n<N, 1, double>(g, tab, cmet, fmet, lam, nu_cell, nu_face,
                                                                        mass, x, y, nbatch, st)));
  }
  return cudaSuccess;
}

// the same operator in FP32 (multigrid levels: metric, sweeps and flux in binary32)
cudaError_t launch_mapped_apply_f32(int n, int ncomp, const LevelGeom& g, const SplitTab& tab, const float* cmet,
                                    const float* fmet, const double* lam, const float* nu_cell, const float* nu_face,
                                    double mass, const float* x, float* y, int nbatch, cudaStream_t st) {
  if (g.ncells == 0 || nbatch == 0) return cudaSuccess;
  if (ncomp == 3) {
    SIPG_MAPPED_DISPATCH(n, return (launch_mapped_apply_n<N, 3, float>(g, tab, cmet, fmet, lam, nu_cell, nu_face,
                                                                       mass, x, y, nbatch, st)));
  } else {
    SIPG_MAPPED_DISPATCH(n, return (launch_mapped_apply_n<N, 1, float>(g, tab, cmet, fmet, lam, nu_cell, nu_face,
                                                                       mass, x, y, nbatch, st)));
  }
  return cudaSuccess;
}

// Vertices of a coarser level of the same structured mesh: every (stride)-th vertex.
__global__ void gather_vertices_kernel(int nxf, int nyf, int nxc, int nyc, int nzc, int stride,
                                       const double* __restrict__ fine, double* __restrict__ coarse) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nv = (int64_t)(nxc + 1) * (nyc + 1) * (nzc + 1);
  if (t >= nv * 3) return;
  const int c = (int)(t % 3);
  const int64_t v = t / 3;
  const int i = (int)(v % (nxc + 1)), j = (int)((v / (nxc + 1)) % (nyc + 1)), k = (int)(v / ((int64_t)(nxc + 1) * (nyc + 1)));
  const int64_t vf = ((int64_t)k * stride * (nyf + 1) + (int64_t)j * stride) * (nxf + 1) + (int64_t)i * stride;
  coarse[t] = fine[vf * 3 + c];
}
cudaError_t launch_gather_vertices(int nxf, int nyf, int nxc, int nyc, int nzc, int stride, const double* fine,
                                   double* coarse, cudaStream_t st) {
  const int64_t n = (int64_t)(nxc + 1) * (nyc + 1) * (nzc + 1) * 3;
  gather_vertices_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(nxf, nyf, nxc, nyc, nzc, stride, fine, coarse);
  return cudaGetLastError();
}

// Diagonal of (mass M + A) on trilinear cells, DoF (c, i) (own-side blocks with
// trial = test = phi_i e_c; g = physical gradient of phi_i, W the point weight):
//  viscous cell:  sum_q W (nu (|g|^2 + g_c^2) + mass phi^2)
//  viscous face:  sum_p W (-nu phi (g.n + n_c g_c) + tau phi^2 (1 + n_c^2)), twice that on a
//                 Dirichlet wall (mirror), nothing on a Neumann wall
//  Poisson:       sum_q W (|g|^2 + mass phi^2);  faces sum_p W (-phi g.n + tau phi^2), x2 on walls
// Face terms reach only the DoFs of the face layer (phi_i vanishes on the face otherwise).
template <int N, int NC>
__global__ void __launch_bounds__(kSplitThreads) mapped_diagonal_kernel(LevelGeom g, SplitTab tab,
                                                                        const double* __restrict__ verts,
                                                                        const double* __restrict__ lam,
                                                                        const double* __restrict__ nu_cell,
                                                                        const double* __restrict__ nu_face,
                                                                        double mass, double* __restrict__ diag) {
  constexpr int N3 = N * N * N, N2 = N * N;
  __shared__ STabSm T;
  __shared__ double X[8][3];
  __shared__ double JI[9][N3], WQ[N3], NU[N3];
  __shared__ double FJ[9][N2], FNm[3][N2], FW[N2], FT[N2], FNU[N2];
  __shared__ double ACC[NC][N3];
  const int e = blockIdx.x;
  load_tab(tab, T);
  load_cell_vertices(g, verts, e, X);
  __syncthreads();
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    const int qx = q % N, qy = (q / N) % N, qz = q / N2;
    double J[3][3], Ji[3][3];
    trilinear_jac(X, tab.gp[qx], tab.gp[qy], tab.gp[qz], J);
    const double det = inverse3(J, Ji);
    for (int m = 0; m < 9; ++m) JI[m][q] = Ji[m / 3][m % 3];
    WQ[q] = T.gw[qx] * T.gw[qy] * T.gw[qz] * det;
    NU[q] = NC == 3 ? nu_cell[(size_t)e * N3 + q] : 1.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N3; i += blockDim.x) {
    const int ix = i % N, iy = (i / N) % N, iz = i / N2;
    double a0 = 0.0, ac[3] = {0.0, 0.0, 0.0}, am = 0.0;
    for (int q = 0; q < N3; ++q) {
      const int qx = q % N, qy = (q / N) % N, qz = q / N2;
      const double sx = T.S[qx * N + ix], sy = T.S[qy * N + iy], sz = T.S[qz * N + iz];
      const double r[3] = {T.DS[qx * N + ix] * sy * sz, sx * T.DS[qy * N + iy] * sz, sx * sy * T.DS[qz * N + iz]};
      double gg[3];
      for (int l = 0; l < 3; ++l) gg[l] = r[0] * JI[l][q] + r[1] * JI[3 + l][q] + r[2] * JI[6 + l][q];
      const double w = WQ[q] * NU[q];
      const double g2 = gg[0] * gg[0] + gg[1] * gg[1] + gg[2] * gg[2];
      a0 += w * g2;
      for (int c = 0; c < 3; ++c) ac[c] += w * gg[c] * gg[c];
      const double ph = sx * sy * sz;
      am += WQ[q] * ph * ph;
    }
    for (int c = 0; c < NC; ++c) ACC[c][i] = a0 + (NC == 3 ? ac[c] : 0.0) + mass * am;
  }
  __syncthreads();
  const double lam_e = lam[e];
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    int t1, t2;
    face_dirs(d, &t1, &t2);
    const int nb = cell_neighbor(g, e, f);
    if (nb < 0 && face_bc(g, e, f) == 1) continue;
    const int fo = 2 * d + (1 - s);
    const double orient = (2.0 * s - 1.0) * (d == 1 ? -1.0 : 1.0);
    const double lam_p = nb >= 0 ? lam[nb] : lam_e;
    const double tau0 = g.cip * (double)(N * N) * fmax(lam_e, lam_p);
    const double mirror = nb >= 0 ? 1.0 : 2.0;
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      double xi[3];
      xi[d] = s ? 1.0 : 0.0;
      xi[t1] = tab.gp[p % N];
      xi[t2] = tab.gp[p / N];
      double J[3][3], Ji[3][3];
      trilinear_jac(X, xi[0], xi[1], xi[2], J);
      inverse3(J, Ji);
      for (int m = 0; m < 9; ++m) FJ[m][p] = Ji[m / 3][m % 3];
      const double ta[3] = {J[0][t1], J[1][t1], J[2][t1]}, tb[3] = {J[0][t2], J[1][t2], J[2][t2]};
      double n[3] = {ta[1] * tb[2] - ta[2] * tb[1], ta[2] * tb[0] - ta[0] * tb[2], ta[0] * tb[1] - ta[1] * tb[0]};
      const double area = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      for (int k = 0; k < 3; ++k) FNm[k][p] = n[k] * orient / area;
      FW[p] = mirror * T.gw[p % N] * T.gw[p / N] * area;
      double nub = 1.0, num = 1.0;
      if (NC == 3) {
        num = nu_face[((size_t)e * 6 + f) * N2 + p];
        const double nup = nb >= 0 ? nu_face[((size_t)nb * 6 + fo) * N2 + p] : num;
        nub = num > nup ? num : nup;
        if (g.face_nu == 1) nub = 0.5 * (num + nup);
        if (g.face_nu == 2) nub = 2.0 * num * nup / (num + nup);
      }
      FNU[p] = num;
      FT[p] = tau0 * nub;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < N2; t += blockDim.x) {
      const int ia = t % N, ib = t / N;
      int idx[3];
      idx[d] = s ? N - 1 : 0;
      idx[t1] = ia;
      idx[t2] = ib;
      const int i = (idx[2] * N + idx[1]) * N + idx[0];
      double acc0 = 0.0, accc[3] = {0.0, 0.0, 0.0};
      for (int p = 0; p < N2; ++p) {
        const int a = p % N, b = p / N;
        const double sa = T.S[a * N + ia], sb = T.S[b * N + ib];
        const double ph = sa * sb;
        double r[3];
        r[d] = T.dS[s][idx[d]] * ph;
        r[t1] = T.DS[a * N + ia] * sb;
        r[t2] = sa * T.DS[b * N + ib];
        double gg[3];
        for (int l = 0; l < 3; ++l) gg[l] = r[0] * FJ[l][p] + r[1] * FJ[3 + l][p] + r[2] * FJ[6 + l][p];
        const double gn = gg[0] * FNm[0][p] + gg[1] * FNm[1][p] + gg[2] * FNm[2][p];
        if (NC == 3) {
          for (int c = 0; c < 3; ++c) {
            const double nc = FNm[c][p];
            accc[c] += FW[p] * (-FNU[p] * ph * (gn + nc * gg[c]) + FT[p] * ph * ph * (1.0 + nc * nc));
          }
        } else {
          acc0 += FW[p] * (-ph * gn + FT[p] * ph * ph);
        }
      }
      for (int c = 0; c < NC; ++c) ACC[c][i] += NC == 3 ? accc[c] : acc0;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < NC * N3; i += blockDim.x) diag[(size_t)e * NC * N3 + i] = ACC[i / N3][i % N3];
}

cudaError_t launch_mapped_diagonal(int n, int ncomp, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                   const double* lam, const double* nu_cell, const double* nu_face, double mass,
                                   double* diag, cudaStream_t st) {
  if (g.ncells == 0) return cudaSuccess;
  if (ncomp == 3) {
    SIPG_MAPPED_DISPATCH(n, (mapped_diagonal_kernel<N, 3><<<g.ncells, kSplitThreads, 0, st>>>(
                                g, tab, verts, lam, nu_cell, nu_face, mass, diag)));
  } else {
    SIPG_MAPPED_DISPATCH(n, (mapped_diagonal_kernel<N, 1><<<g.ncells, kSplitThreads, 0, st>>>(
                                g, tab, verts, lam, nu_cell, nu_face, mass, diag)));
  }
  return cudaGetLastError();
}

cudaError_t launch_mapped_lambda(int n, const LevelGeom& g, const SplitTab& tab, const double* verts, double* lam,
                                 cudaStream_t st) {
  if (g.ncells == 0) return cudaSuccess;
  mapped_lambda_kernel<<<(g.ncells + 127) / 128, 128, 0, st>>>(g, tab, n, verts, lam);
  return cudaGetLastError();
}

cudaError_t launch_mapped_viscosity(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                    const RheologyDev& rh, const double* u, double* nu_cell, double* nu_face,
                                    cudaStream_t st) {
  if (g.ncells == 0) return cudaSuccess;
  SIPG_MAPPED_DISPATCH(n, (mapped_viscosity_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(
                              g, tab, verts, rh, u, nu_cell, nu_face)));
  return cudaGetLastError();
}

}  // namespace sipg
