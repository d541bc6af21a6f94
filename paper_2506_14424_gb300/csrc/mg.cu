// Multigrid and Krylov building blocks: operator diagonal, p/h transfers,
// Chebyshev and CG vector updates, deterministic reductions and the dense FP64
// coarse-level helpers (Sec. 5.4 of the paper).
#include "ff.cuh"
#include "kernels.cuh"

#include <algorithm>

namespace sipg {

namespace {
constexpr int kBS = 256;
inline int blocks_for(int64_t n) { return (int)std::min<int64_t>((n + kBS - 1) / kBS, 152 * 16); }
}  // namespace

// ---------------------------------------------------------------- diagonal
// Diagonal of (m M + A) for DoF (c, i) of a cell: the cell integral of the
// test function against itself plus the own-side face terms (trial = test on
// the own side, zero neighbour state on interior faces, mirror state on
// Dirichlet faces). With n = sigma e_d and phi the scalar shape function:
//  viscous cell:  sum_q W nu (|grad phi|^2 + (d_c phi)^2) + m W phi^2
//  viscous face:  interior  -nu sigma phi d_d phi (1 + delta_cd) + tau phi^2 (1 + delta_cd)
//                 Dirichlet 2 x the same with tau of the wall
//  Poisson cell:  sum_q W |grad phi|^2 + m W phi^2
//  Poisson face:  interior  -sigma phi d_d phi + tau phi^2;  Dirichlet 2 x the same
// The cell sums factor over the tensor product: sum_q F(q) prod_d A_d[q_d][i_d]^2
// with F = W nu (or W) and A_d = DS (derivative direction) or S, one sweep per
// direction; face terms vanish unless the DoF lies on the face layer, and
// there they reduce to 2D contractions with S^2 (one per face).
// One CTA per cell.
template <int N, int NC>
__global__ void diagonal_kernel(LevelGeom g, Tab tab, const double* __restrict__ nu_cell,
                                const double* __restrict__ nu_face, double mass, double* __restrict__ diag,
                                bool interior_faces) {
  constexpr int N2 = N * N, N3 = N2 * N;
  __shared__ double F[N3], Fm[N3], T1[N3], T2[N3], C[4][N3];
  __shared__ double S2[N2], D2[N2], FD[6][N2];
  const int e = blockIdx.x;
  const double detJ = g.h[0] * g.h[1] * g.h[2];
  for (int i = threadIdx.x; i < N2; i += blockDim.x) {
    S2[i] = tab.S[i] * tab.S[i];
    D2[i] = tab.DS[i] * tab.DS[i];
  }
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    const double W = tab.gw[q % N] * tab.gw[(q / N) % N] * tab.gw[q / N2] * detJ;
    F[q] = NC == 3 ? W * nu_cell[(size_t)e * N3 + q] : W;
    Fm[q] = mass * W;
  }
  __syncthreads();
  // C[l] (l = 0, 1, 2: derivative direction l; l = 3: mass) by three sweeps
  for (int l = 0; l < 4; ++l) {
    const double* src = l < 3 ? F : Fm;
    const double* Ax = l == 0 ? D2 : S2;
    const double* Ay = l == 1 ? D2 : S2;
    const double* Az = l == 2 ? D2 : S2;
    for (int o = threadIdx.x; o < N3; o += blockDim.x) {  // (qz, qy, ix)
      const int ix = o % N, qy = (o / N) % N, qz = o / N2;
      double s = 0.0;
      for (int qx = 0; qx < N; ++qx) s += Ax[qx * N + ix] * src[(qz * N + qy) * N + qx];
      T1[o] = s;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < N3; o += blockDim.x) {  // (qz, iy, ix)
      const int ix = o % N, iy = (o / N) % N, qz = o / N2;
      double s = 0.0;
      for (int qy = 0; qy < N; ++qy) s += Ay[qy * N + iy] * T1[(qz * N + qy) * N + ix];
      T2[o] = s;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < N3; o += blockDim.x) {  // (iz, iy, ix)
      const int ix = o % N, iy = (o / N) % N, iz = o / N2;
      double s = 0.0;
      for (int qz = 0; qz < N; ++qz) s += Az[qz * N + iz] * T2[(qz * N + iy) * N + ix];
      C[l][o] = s;
    }
    __syncthreads();
  }
  // faces: both face terms are proportional to phi_i(p)^2 (d_d phi_i = l'(layer) phi_i / h_d
  // on the face), so each face is a 2D contraction of a per-point factor with S^2:
  //   FD_f[a_i, b_i] = sum_{a,b} S[a][a_i]^2 S[b][b_i]^2 F_f(a, b)
  const double lam_e = penalty_lambda(g, e);
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    const int nb = cell_neighbor(g, e, f);
    const bool skip = (nb < 0 && face_bc(g, e, f) == 1)      // homogeneous Neumann: no face term
                      || (nb >= 0 && !interior_faces);  // continuous level: jumps vanish
    const double sigma = s ? 1.0 : -1.0;
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const double lam = nb >= 0 ? fmax(lam_e, penalty_lambda(g, nb)) : lam_e;
    const double dl = (s ? tab.dS1[N - 1] : tab.dS0[0]) * g.ih[d];  // l'(layer) / h_d
    const double area = g.h[t1] * g.h[t2];
    const double mirror = nb >= 0 ? 1.0 : 2.0;
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      const double W = tab.gw[p % N] * tab.gw[p / N] * area;
      double v = 0.0;
      if (!skip) {
        if (NC == 3) {
          const double num = nu_face[((size_t)e * 6 + f) * N2 + p];
          const double nup = nb >= 0 ? nu_face[((size_t)nb * 6 + (f ^ 1)) * N2 + p] : num;
          double nub = num > nup ? num : nup;
          if (g.face_nu == 1) nub = 0.5 * (num + nup);
          if (g.face_nu == 2) nub = 2.0 * num * nup / (num + nup);
          const double tau = g.cip * N * N * lam * nub;
          v = mirror * W * (-num * sigma * dl + tau);
        } else {
          const double tau = g.cip * N * N * lam;
          v = mirror * W * (-sigma * dl + tau);
        }
      }
      T1[p] = v;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < N2; o += blockDim.x) {  // (b, a_i)
      const int ai = o % N, bq = o / N;
      double acc = 0.0;
      for (int aq = 0; aq < N; ++aq) acc += S2[aq * N + ai] * T1[bq * N + aq];
      T2[o] = acc;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < N2; o += blockDim.x) {  // (b_i, a_i)
      const int ai = o % N, bi = o / N;
      double acc = 0.0;
      for (int bq = 0; bq < N; ++bq) acc += S2[bq * N + bi] * T2[bq * N + ai];
      FD[f][o] = acc;
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < NC * N3; idx += blockDim.x) {
    const int c = idx / N3, r = idx % N3;
    const int ii[3] = {r % N, (r / N) % N, r / N2};
    double acc = C[3][r];
    for (int l = 0; l < 3; ++l) {
      const double f = (NC == 3 && l == c) ? 2.0 : 1.0;
      acc += f * g.ih[l] * g.ih[l] * C[l][r];
    }
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1, s = f & 1;
      if (ii[d] != (s ? N - 1 : 0)) continue;  // shape function vanishes on this face
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      const double fac = (NC == 3 && c == d) ? 2.0 : 1.0;
      acc += fac * FD[f][ii[t1] + N * ii[t2]];
    }
    diag[((size_t)e * NC + c) * N3 + r] = acc;
  }
}

cudaError_t launch_diagonal(int n, int ncomp, const LevelGeom& g, const Tab& tab, const double* nu_cell,
                            const double* nu_face, double mass, double* diag, cudaStream_t st,
                            bool interior_faces) {
  if (g.ncells == 0) return cudaSuccess;
#define SIPG_DIAG(NN)                                                                              \
  case NN:                                                                                         \
    if (ncomp == 3)                                                                                \
      diagonal_kernel<NN, 3><<<g.ncells, 128, 0, st>>>(g, tab, nu_cell, nu_face, mass, diag, interior_faces); \
    else                                                                                           \
      diagonal_kernel<NN, 1><<<g.ncells, 128, 0, st>>>(g, tab, nu_cell, nu_face, mass, diag, interior_faces); \
    break;
  switch (n) {
    SIPG_DIAG(2) SIPG_DIAG(3) SIPG_DIAG(4) SIPG_DIAG(5) SIPG_DIAG(6)
    default: return cudaErrorInvalidValue;
  }
#undef SIPG_DIAG
  return cudaGetLastError();
}

// --------------------------------------------------------------- transfers
// p-transfer on one cell and component: fine = (E x E x E) coarse with
// E[i*nc + j] = l^coarse_j(xi^fine_i) (prolongation, dir +1), or the
// transpose (restriction, dir -1). One thread per output value; the 1D
// weights are staged in shared memory in the vector's precision.
template <typename T>
__global__ void p_transfer_kernel(int nf, int nc, int ntens, TransferTab tt, int dir, const T* __restrict__ in,
                                  T* __restrict__ out) {
  __shared__ T E[kMaxN * kMaxN];
  for (int i = threadIdx.x; i < nf * nc; i += blockDim.x) E[i] = T(tt.E[i]);
  __syncthreads();
  const int nin = dir > 0 ? nc : nf, nout = dir > 0 ? nf : nc;
  const int in3 = nin * nin * nin, out3 = nout * nout * nout;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)ntens * out3) return;
  const int t = (int)(idx / out3), r = (int)(idx % out3);
  const int o[3] = {r % nout, (r / nout) % nout, r / (nout * nout)};
  const T* src = in + (size_t)t * in3;
  T acc = T(0);
  for (int k = 0; k < nin; ++k) {
    const T ez = dir > 0 ? E[o[2] * nc + k] : E[k * nc + o[2]];
    for (int j = 0; j < nin; ++j) {
      const T ezy = ez * (dir > 0 ? E[o[1] * nc + j] : E[j * nc + o[1]]);
      const T* row = src + (k * nin + j) * nin;
      T s = T(0);
      for (int i = 0; i < nin; ++i) s += (dir > 0 ? E[o[0] * nc + i] : E[i * nc + o[0]]) * row[i];
      acc += ezy * s;
    }
  }
  out[idx] = acc;
}

template <typename T>
cudaError_t launch_p_transfer(int nf, int nc, int ncomp, int ncells, const TransferTab& tt, int dir,
                              const T* in, T* out, cudaStream_t st) {
  const int nout = dir > 0 ? nf : nc;
  const int64_t total = (int64_t)ncells * ncomp * nout * nout * nout;
  const int blocks = (int)((total + kBS - 1) / kBS);
  if (blocks == 0) return cudaSuccess;
  p_transfer_kernel<T><<<blocks, kBS, 0, st>>>(nf, nc, ncells * ncomp, tt, dir, in, out);
  return cudaGetLastError();
}

// h-transfer: coarse cell -> its 8 children on the once-refined mesh; child
// (cx, cy, cz) uses E_c[i*n + j] = l_j((xi_i + c)/2). Prolongation: one thread
// per fine value; restriction: one thread per coarse value summing its children.
template <typename T>
__global__ void h_prolong_kernel(int n, int ncomp, LevelGeom fine, LevelGeom coarse, TransferTab tt,
                                 const T* __restrict__ in, T* __restrict__ out) {
  __shared__ T E0[kMaxN * kMaxN], E1[kMaxN * kMaxN];
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    E0[i] = T(tt.E[i]);
    E1[i] = T(tt.E1[i]);
  }
  __syncthreads();
  const int n3 = n * n * n;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)fine.ncells * ncomp * n3) return;
  const int ef = (int)(idx / (ncomp * n3));
  const int rem = (int)(idx % (ncomp * n3));
  const int comp = rem / n3, r = rem % n3;
  int fi[3];
  cell_ijk(fine, ef, fi);
  const int fx = fi[0], fy = fi[1], fz = fi[2];
  const int ec = grid_cell(coarse, fx / 2, fy / 2, fz / 2);
  const T* Ex = (fx & 1) ? E1 : E0;
  const T* Ey = (fy & 1) ? E1 : E0;
  const T* Ez = (fz & 1) ? E1 : E0;
  const int o[3] = {r % n, (r / n) % n, r / (n * n)};
  const T* src = in + ((size_t)ec * ncomp + comp) * n3;
  T acc = T(0);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j) {
      const T wzy = Ez[o[2] * n + k] * Ey[o[1] * n + j];
      T s = T(0);
      for (int i = 0; i < n; ++i) s += Ex[o[0] * n + i] * src[(k * n + j) * n + i];
      acc += wzy * s;
    }
  out[idx] = acc;
}

template <typename T>
__global__ void h_restrict_kernel(int n, int ncomp, LevelGeom fine, LevelGeom coarse, TransferTab tt,
                                  const T* __restrict__ in, T* __restrict__ out) {
  __shared__ T E0[kMaxN * kMaxN], E1[kMaxN * kMaxN];
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    E0[i] = T(tt.E[i]);
    E1[i] = T(tt.E1[i]);
  }
  __syncthreads();
  const int n3 = n * n * n;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)coarse.ncells * ncomp * n3) return;
  const int ec = (int)(idx / (ncomp * n3));
  const int rem = (int)(idx % (ncomp * n3));
  const int comp = rem / n3, r = rem % n3;
  int ci[3];
  cell_ijk(coarse, ec, ci);
  const int cx = ci[0], cy = ci[1], cz = ci[2];
  const int o[3] = {r % n, (r / n) % n, r / (n * n)};
  T acc = T(0);
  for (int ch = 0; ch < 8; ++ch) {
    const int bx = ch & 1, by = (ch >> 1) & 1, bz = ch >> 2;
    const int ef = grid_cell(fine, 2 * cx + bx, 2 * cy + by, 2 * cz + bz);
    const T* Ex = bx ? E1 : E0;
    const T* Ey = by ? E1 : E0;
    const T* Ez = bz ? E1 : E0;
    const T* src = in + ((size_t)ef * ncomp + comp) * n3;
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j) {
        const T wzy = Ez[k * n + o[2]] * Ey[j * n + o[1]];
        T s = T(0);
        for (int i = 0; i < n; ++i) s += Ex[i * n + o[0]] * src[(k * n + j) * n + i];
        acc += wzy * s;
      }
  }
  out[idx] = acc;
}

template <typename T>
cudaError_t launch_h_transfer(int n, int ncomp, const LevelGeom& fine, const LevelGeom& coarse,
                              const TransferTab& tt, int dir, const T* in, T* out, cudaStream_t st) {
  const int64_t total = (int64_t)(dir > 0 ? fine.ncells : coarse.ncells) * ncomp * n * n * n;
  const int blocks = (int)((total + kBS - 1) / kBS);
  if (blocks == 0) return cudaSuccess;
  if (dir > 0)
    h_prolong_kernel<T><<<blocks, kBS, 0, st>>>(n, ncomp, fine, coarse, tt, in, out);
  else
    h_restrict_kernel<T><<<blocks, kBS, 0, st>>>(n, ncomp, fine, coarse, tt, in, out);
  return cudaGetLastError();
}

// Downward interpolation of the linearization velocity (nodal values of the
// fine function at the coarse nodes).
__global__ void p_interp_down_kernel(int nf, int nc, int ntens, TransferTab tt, const double* __restrict__ in,
                                     double* __restrict__ out) {
  const int f3 = nf * nf * nf, c3 = nc * nc * nc;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)ntens * c3) return;
  const int t = (int)(idx / c3), r = (int)(idx % c3);
  const int o[3] = {r % nc, (r / nc) % nc, r / (nc * nc)};
  const double* src = in + (size_t)t * f3;
  double acc = 0.0;
  for (int k = 0; k < nf; ++k)
    for (int j = 0; j < nf; ++j)
      for (int i = 0; i < nf; ++i)
        acc += tt.E[o[0] * nf + i] * tt.E[o[1] * nf + j] * tt.E[o[2] * nf + k] * src[(k * nf + j) * nf + i];
  out[idx] = acc;
}

cudaError_t launch_p_interp_down(int nf, int nc, int ncomp, int ncells, const TransferTab& tt,
                                 const double* in, double* out, cudaStream_t st) {
  const int64_t total = (int64_t)ncells * ncomp * nc * nc * nc;
  const int blocks = (int)((total + kBS - 1) / kBS);
  if (blocks == 0) return cudaSuccess;
  p_interp_down_kernel<<<blocks, kBS, 0, st>>>(nf, nc, ncells * ncomp, tt, in, out);
  return cudaGetLastError();
}

struct ChildMap { int c[kMaxN]; };

__global__ void h_interp_down_kernel(int n, int ncomp, LevelGeom fine, LevelGeom coarse, TransferTab tt,
                                     ChildMap cm, const double* __restrict__ in, double* __restrict__ out) {
  const int n3 = n * n * n;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)coarse.ncells * ncomp * n3) return;
  const int ec = (int)(idx / (ncomp * n3));
  const int rem = (int)(idx % (ncomp * n3));
  const int comp = rem / n3, r = rem % n3;
  int ci[3];
  cell_ijk(coarse, ec, ci);
  const int o[3] = {r % n, (r / n) % n, r / (n * n)};
  const int ef = grid_cell(fine, 2 * ci[0] + cm.c[o[0]], 2 * ci[1] + cm.c[o[1]], 2 * ci[2] + cm.c[o[2]]);
  const double* src = in + ((size_t)ef * ncomp + comp) * n3;
  double acc = 0.0;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i)
        acc += tt.E[o[0] * n + i] * tt.E[o[1] * n + j] * tt.E[o[2] * n + k] * src[(k * n + j) * n + i];
  out[idx] = acc;
}

cudaError_t launch_h_interp_down(int n, int ncomp, const LevelGeom& fine, const LevelGeom& coarse,
                                 const TransferTab& tt, const int* child, const double* in, double* out,
                                 cudaStream_t st) {
  ChildMap cm{};
  for (int i = 0; i < n; ++i) cm.c[i] = child[i];
  const int64_t total = (int64_t)coarse.ncells * ncomp * n * n * n;
  const int blocks = (int)((total + kBS - 1) / kBS);
  if (blocks == 0) return cudaSuccess;
  h_interp_down_kernel<<<blocks, kBS, 0, st>>>(n, ncomp, fine, coarse, tt, cm, in, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------ vector updates
template <typename T>
__global__ void axpby_kernel(int64_t n, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
template <typename T>
cudaError_t launch_axpby(int64_t n, T a, const T* x, T b, T* y, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  axpby_kernel<T><<<blocks_for(n), kBS, 0, st>>>(n, a, x, b, y);
  return cudaGetLastError();
}

template <typename T>
__global__ void sub_kernel(int64_t n, const T* __restrict__ b, const T* __restrict__ t, T* __restrict__ r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - t[i];
}
template <typename T>
cudaError_t launch_sub(int64_t n, const T* b, const T* t, T* r, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  sub_kernel<T><<<blocks_for(n), kBS, 0, st>>>(n, b, t, r);
  return cudaGetLastError();
}

template <typename T>
__global__ void cheb_kernel(int64_t n, T c1, T c2, const T* __restrict__ dinv, const T* __restrict__ b,
                            const T* __restrict__ t, T* __restrict__ d, T* __restrict__ x, bool first_zero) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T r = t ? b[i] - t[i] : b[i];
    const T dn = (first_zero ? T(0) : c1 * d[i]) + c2 * dinv[i] * r;
    d[i] = dn;
    x[i] = first_zero ? dn : x[i] + dn;
  }
}
template <typename T>
cudaError_t launch_cheb(int64_t n, T c1, T c2, const T* dinv, const T* b, const T* t, T* d, T* x, bool x_zero,
                        cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  cheb_kernel<T><<<blocks_for(n), kBS, 0, st>>>(n, c1, c2, dinv, b, t, d, x, x_zero);
  return cudaGetLastError();
}

template <typename S, typename D>
__global__ void cast_kernel(int64_t n, const S* __restrict__ in, D* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = D(in[i]);
}
template <typename S, typename D>
cudaError_t launch_cast(int64_t n, const S* in, D* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  cast_kernel<S, D><<<blocks_for(n), kBS, 0, st>>>(n, in, out);
  return cudaGetLastError();
}

template <typename T>
__global__ void fill_kernel(int64_t n, T v, T* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v;
}
template <typename T>
cudaError_t launch_fill(int64_t n, T v, T* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  fill_kernel<T><<<blocks_for(n), kBS, 0, st>>>(n, v, out);
  return cudaGetLastError();
}

__global__ void add_scaled_kernel(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}
cudaError_t launch_add_scaled_f64(int64_t n, double a, const double* x, double* y, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  add_scaled_kernel<<<blocks_for(n), kBS, 0, st>>>(n, a, x, y);
  return cudaGetLastError();
}

__global__ void mul_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] * b[i];
}
cudaError_t launch_mul(int64_t n, const double* a, const double* b, double* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  mul_kernel<<<blocks_for(n), kBS, 0, st>>>(n, a, b, out);
  return cudaGetLastError();
}

__global__ void reciprocal_kernel(int64_t n, const double* __restrict__ a, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = 1.0 / a[i];
}
cudaError_t launch_reciprocal(int64_t n, const double* a, double* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  reciprocal_kernel<<<blocks_for(n), kBS, 0, st>>>(n, a, out);
  return cudaGetLastError();
}
__global__ void scale_kernel(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}
cudaError_t launch_scale(int64_t n, double a, const double* x, double* y, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  scale_kernel<<<blocks_for(n), kBS, 0, st>>>(n, a, x, y);
  return cudaGetLastError();
}

__global__ void sqrt_kernel(int64_t n, double* v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = sqrt(v[i]);
}
cudaError_t launch_sqrt(int64_t n, double* v, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  sqrt_kernel<<<blocks_for(n), kBS, 0, st>>>(n, v);
  return cudaGetLastError();
}

// Counter-based uniform(-1, 1) numbers (splitmix64 of seed + index).
__global__ void random_kernel(int64_t n, uint64_t seed, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    out[i] = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
  }
}
cudaError_t launch_random(int64_t n, uint64_t seed, double* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  random_kernel<<<blocks_for(n), kBS, 0, st>>>(n, seed, out);
  return cudaGetLastError();
}

// Deterministic reductions: fixed grid, fixed per-thread order, tree in shared.
template <bool DOT>
__global__ void partial_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                               double* __restrict__ partials) {
  __shared__ double red[kBS];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kBS + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kBS)
    s += DOT ? a[i] * b[i] : a[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kBS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}
__global__ void final_kernel(const double* __restrict__ partials, double* __restrict__ out) {
  __shared__ double red[512];
  red[threadIdx.x] = threadIdx.x < kDotBlocks ? partials[threadIdx.x] : 0.0;
  __syncthreads();
  for (int w = 256; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}
cudaError_t launch_dot(int64_t n, const double* a, const double* b, double* partials, double* dev_out,
                       cudaStream_t st) {
  partial_kernel<true><<<kDotBlocks, kBS, 0, st>>>(n, a, b, partials);
  final_kernel<<<1, 512, 0, st>>>(partials, dev_out);
  return cudaGetLastError();
}
cudaError_t launch_sum(int64_t n, const double* a, double* partials, double* dev_out, cudaStream_t st) {
  partial_kernel<false><<<kDotBlocks, kBS, 0, st>>>(n, a, nullptr, partials);
  final_kernel<<<1, 512, 0, st>>>(partials, dev_out);
  return cudaGetLastError();
}

// y += scale * c[0] (c on the device), used for mean removal.
__global__ void add_const_kernel(int64_t n, const double* __restrict__ c, double scale, double* __restrict__ y) {
  const double v = scale * c[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += v;
}
cudaError_t launch_add_const(int64_t n, const double* dev_c, double scale, double* y, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  add_const_kernel<<<blocks_for(n), kBS, 0, st>>>(n, dev_c, scale, y);
  return cudaGetLastError();
}

__global__ void finite_kernel(int64_t n, const double* __restrict__ a, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(a[i])) *flag = 1;
}
cudaError_t launch_check_finite(int64_t n, const double* a, int* flag, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  finite_kernel<<<blocks_for(n), kBS, 0, st>>>(n, a, flag);
  return cudaGetLastError();
}

// ----------------------------------------------------------- dense coarse
// Columns j0 .. j0+ncols-1 of the N x N identity, stored column-major.
__global__ void unit_columns_kernel(int N, int j0, int ncols, double* out) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)N * ncols) return;
  const int col = (int)(idx / N), row = (int)(idx % N);
  out[idx] = row == j0 + col ? 1.0 : 0.0;
}
cudaError_t launch_unit_columns(int N, int j0, int ncols, double* out, cudaStream_t st) {
  const int64_t total = (int64_t)N * ncols;
  unit_columns_kernel<<<(int)((total + kBS - 1) / kBS), kBS, 0, st>>>(N, j0, ncols, out);
  return cudaGetLastError();
}

// Columns of a DG operator by colouring: probe vector b = (colour, local DoF l)
// is 1 at DoF l of every cell of that colour; since the closed face
// neighbourhoods of the cells of one colour are disjoint, row r of A probe_b
// belongs to the column of the unique cell of that colour in the neighbourhood
// of r's cell (owner table), or is zero.
__global__ void colour_probe_kernel(int N, int dpc, int nb, const int* __restrict__ colour, double* __restrict__ out) {
  const int64_t total = (int64_t)N * nb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / N), r = (int)(i - (int64_t)b * N);
    out[i] = (colour[r / dpc] == b / dpc && r % dpc == b % dpc) ? 1.0 : 0.0;
  }
}
__global__ void colour_scatter_kernel(int N, int C, int dpc, int nb, const int* __restrict__ owner,
                                      const double* __restrict__ Y, double* __restrict__ A) {
  const int64_t total = (int64_t)N * nb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / N), r = (int)(i - (int64_t)b * N);
    const int c = owner[(size_t)(b / dpc) * C + r / dpc];
    if (c >= 0) A[((size_t)c * dpc + b % dpc) * N + r] = Y[i];
  }
}
cudaError_t launch_colour_probes(int N, int dpc, int nb, const int* colour, double* out, cudaStream_t st) {
  const int64_t total = (int64_t)N * nb;
  colour_probe_kernel<<<(int)std::min<int64_t>((total + kBS - 1) / kBS, 152 * 32), kBS, 0, st>>>(N, dpc, nb, colour,
                                                                                                out);
  return cudaGetLastError();
}
cudaError_t launch_colour_scatter(int N, int C, int dpc, int nb, const int* owner, const double* Y, double* A,
                                  cudaStream_t st) {
  const int64_t total = (int64_t)N * nb;
  colour_scatter_kernel<<<(int)std::min<int64_t>((total + kBS - 1) / kBS, 152 * 32), kBS, 0, st>>>(N, C, dpc, nb,
                                                                                                  owner, Y, A);
  return cudaGetLastError();
}

// Gauss-Jordan inverse of the dense coarse matrix (no pivoting: the coarse
// operator is SPD, or SPD after the rank-one term of the singular Poisson
// case), entries in float-float (float2 = (hi, lo)) for the FP32 pipe.
// Blocked Gauss-Jordan: pivots k0 .. k0+b-1 at once (b <= 16). With P = A[K,K],
// R = P^-1 A[K,:]:  new[K,K] = P^-1, new[K,j] = R[.,j], new[i,K] = -A[i,K] P^-1,
// new[i,j] = A[i,j] - A[i,K] R[.,j]  (b = 1 is the step above).
constexpr int kGjBlock = 16;
__global__ void gj_block_inv_kernel(int N, int k0, int b, const float2* __restrict__ A, float2* __restrict__ Pinv) {
  __shared__ ff M[kGjBlock][kGjBlock], I[kGjBlock][kGjBlock];
  const int t = threadIdx.x, ti = t / b, tj = t % b;
  const bool act = t < b * b;
  if (act) {
    const float2 v = A[(size_t)(k0 + ti) * N + k0 + tj];
    M[ti][tj] = ff(v.x, v.y);
    I[ti][tj] = ff(ti == tj ? 1.0f : 0.0f);
  }
  for (int p = 0; p < b; ++p) {
    __syncthreads();
    const ff inv = ff(1.0f) / M[p][p];
    const ff fac = act ? M[ti][p] : ff(0.0f);
    __syncthreads();
    if (act && ti == p) {
      M[p][tj] = M[p][tj] * inv;
      I[p][tj] = I[p][tj] * inv;
    }
    __syncthreads();
    if (act && ti != p) {
      M[ti][tj] = M[ti][tj] - fac * M[p][tj];
      I[ti][tj] = I[ti][tj] - fac * I[p][tj];
    }
  }
  __syncthreads();
  if (act) Pinv[ti * b + tj] = make_float2(I[ti][tj].hi, I[ti][tj].lo);
}
__global__ void gj_block_r_kernel(int N, int k0, int b, const float2* __restrict__ A, const float2* __restrict__ Pinv,
                                  float2* __restrict__ R) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  ff col[kGjBlock];
  for (int l = 0; l < b; ++l) {
    const float2 v = A[(size_t)(k0 + l) * N + j];
    col[l] = ff(v.x, v.y);
  }
  for (int m = 0; m < b; ++m) {
    Acc<ff> acc;
    for (int l = 0; l < b; ++l) {
      const float2 pv = Pinv[m * b + l];
      acc.add(ff(pv.x, pv.y), col[l]);
    }
    const ff r = acc.get();
    R[(size_t)m * N + j] = make_float2(r.hi, r.lo);
  }
}
__global__ void gj_block_update_kernel(int N, int k0, int b, const float2* __restrict__ A,
                                       const float2* __restrict__ Pinv, const float2* __restrict__ R,
                                       float2* __restrict__ B) {
  __shared__ ff rowK[kGjBlock];
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (threadIdx.x < b) {
    const float2 v = A[(size_t)i * N + k0 + threadIdx.x];
    rowK[threadIdx.x] = ff(v.x, v.y);
  }
  __syncthreads();
  if (j >= N) return;
  const bool ik = i >= k0 && i < k0 + b, jk = j >= k0 && j < k0 + b;
  ff v;
  if (ik && jk) {
    const float2 p = Pinv[(i - k0) * b + (j - k0)];
    v = ff(p.x, p.y);
  } else if (ik) {
    const float2 r = R[(size_t)(i - k0) * N + j];
    v = ff(r.x, r.y);
  } else if (jk) {
    Acc<ff> acc;
    for (int m = 0; m < b; ++m) {
      const float2 p = Pinv[m * b + (j - k0)];
      acc.add(rowK[m], ff(p.x, p.y));
    }
    v = -acc.get();
  } else {
    Acc<ff> acc;
    for (int m = 0; m < b; ++m) {
      const float2 r = R[(size_t)m * N + j];
      acc.add(rowK[m], ff(r.x, r.y));
    }
    const float2 a = A[(size_t)i * N + j];
    v = ff(a.x, a.y) - acc.get();
  }
  B[(size_t)i * N + j] = make_float2(v.hi, v.lo);
}
cudaError_t launch_gj_block(int N, int k0, int b, const float2* A, float2* B, float2* Pinv, float2* R,
                            cudaStream_t st) {
  if (b < 1 || b > kGjBlock) return cudaErrorInvalidValue;
  gj_block_inv_kernel<<<1, kGjBlock * kGjBlock, 0, st>>>(N, k0, b, A, Pinv);
  gj_block_r_kernel<<<(N + kBS - 1) / kBS, kBS, 0, st>>>(N, k0, b, A, Pinv, R);
  gj_block_update_kernel<<<dim3((N + kBS - 1) / kBS, N), kBS, 0, st>>>(N, k0, b, A, Pinv, R, B);
  return cudaGetLastError();
}

// in-place binary64 <-> float-float (same 8 bytes per entry)
__global__ void to_ff_kernel(int64_t n, double* v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const ff a(v[i]);
    reinterpret_cast<float2*>(v)[i] = make_float2(a.hi, a.lo);
  }
}
__global__ void from_ff_kernel(int64_t n, double* v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = reinterpret_cast<const float2*>(v)[i];
    v[i] = to_double(ff(a.x, a.y));
  }
}
cudaError_t launch_to_ff_inplace(int64_t n, double* v, cudaStream_t st) {
  to_ff_kernel<<<blocks_for(n), kBS, 0, st>>>(n, v);
  return cudaGetLastError();
}
cudaError_t launch_from_ff_inplace(int64_t n, double* v, cudaStream_t st) {
  from_ff_kernel<<<blocks_for(n), kBS, 0, st>>>(n, v);
  return cudaGetLastError();
}

// y = M x, M row-major N x N: one warp per row.
__global__ void gemv_kernel(int N, const double* __restrict__ M, const double* __restrict__ x, double* __restrict__ y) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  double s = 0.0;
  for (int j = lane; j < N; j += 32) s += M[(size_t)row * N + j] * x[j];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) y[row] = s;
}
cudaError_t launch_gemv(int N, const double* M, const double* x, double* y, cudaStream_t st) {
  gemv_kernel<<<(N + 7) / 8, 256, 0, st>>>(N, M, x, y);
  return cudaGetLastError();
}

__global__ void add_rank1_kernel(int N, double c, double* M) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < (int64_t)N * N) M[idx] += c;
}
cudaError_t launch_add_rank1(int N, double c, double* M, cudaStream_t st) {
  const int64_t total = (int64_t)N * N;
  add_rank1_kernel<<<(int)((total + kBS - 1) / kBS), kBS, 0, st>>>(N, c, M);
  return cudaGetLastError();
}

// explicit instantiations
#define SIPG_INST(T)                                                                                      \
  template cudaError_t launch_p_transfer<T>(int, int, int, int, const TransferTab&, int, const T*, T*,   \
                                            cudaStream_t);                                              \
  template cudaError_t launch_h_transfer<T>(int, int, const LevelGeom&, const LevelGeom&,                \
                                            const TransferTab&, int, const T*, T*, cudaStream_t);        \
  template cudaError_t launch_axpby<T>(int64_t, T, const T*, T, T*, cudaStream_t);                       \
  template cudaError_t launch_sub<T>(int64_t, const T*, const T*, T*, cudaStream_t);                     \
  template cudaError_t launch_cheb<T>(int64_t, T, T, const T*, const T*, const T*, T*, T*, bool,         \
                                      cudaStream_t);                                                     \
  template cudaError_t launch_fill<T>(int64_t, T, T*, cudaStream_t);
SIPG_INST(double)
SIPG_INST(float)
#undef SIPG_INST
template cudaError_t launch_cast<double, float>(int64_t, const double*, float*, cudaStream_t);
template cudaError_t launch_cast<float, double>(int64_t, const float*, double*, cudaStream_t);
template cudaError_t launch_cast<double, double>(int64_t, const double*, double*, cudaStream_t);

}  // namespace sipg
