// Generic shared-memory tensor sweeps and the split-step tables in shared
// memory, used by the splitting-step forms (split.cu) and by the operators on
// trilinear cells (mapped.cu). Device code only; one CTA per cell, the CTA's
// threads share each sweep's outputs.
#pragma once
#include "common.cuh"

namespace sipg {
namespace sweeps {

constexpr int kSplitThreads = 128;

// out = A along DIR applied to the tensor in (extents EX, EY, EZ, x fastest);
// A row-major [NO][E_DIR] (TR = false) or [E_DIR][NO] (TR = true), leading dim lda
template <int EX, int EY, int EZ, int DIR, int NO, bool TR, typename R>
__device__ __forceinline__ void sweep(const R* A, int lda, const R* in, R* out) {
  constexpr int OX = DIR == 0 ? NO : EX, OY = DIR == 1 ? NO : EY, OZ = DIR == 2 ? NO : EZ;
  constexpr int EIN = DIR == 0 ? EX : (DIR == 1 ? EY : EZ);
  constexpr int SIN = DIR == 0 ? 1 : (DIR == 1 ? EX : EX * EY);
  for (int t = threadIdx.x; t < OX * OY * OZ; t += blockDim.x) {
    const int x = t % OX, y = (t / OX) % OY, z = t / (OX * OY);
    const int o = DIR == 0 ? x : (DIR == 1 ? y : z);
    const int base = (DIR == 0 ? 0 : x) + (DIR == 1 ? 0 : y) * EX + (DIR == 2 ? 0 : z) * EX * EY;
    R acc = R(0);
#pragma unroll
    for (int m = 0; m < EIN; ++m) acc += (TR ? A[m * lda + o] : A[o * lda + m]) * in[base + m * SIN];
    out[t] = acc;
  }
}

// the same on ntens tensors stored one after another (inputs EX*EY*EZ apart,
// outputs OX*OY*OZ apart): several cells of a CTA in one pass
template <int EX, int EY, int EZ, int DIR, int NO, bool TR, typename R>
__device__ __forceinline__ void sweepb(const R* A, int lda, const R* in, R* out, int ntens) {
  constexpr int OX = DIR == 0 ? NO : EX, OY = DIR == 1 ? NO : EY, OZ = DIR == 2 ? NO : EZ;
  constexpr int EIN = DIR == 0 ? EX : (DIR == 1 ? EY : EZ);
  constexpr int SIN = DIR == 0 ? 1 : (DIR == 1 ? EX : EX * EY);
  constexpr int SI = EX * EY * EZ, SO = OX * OY * OZ;
  for (int t = threadIdx.x; t < ntens * SO; t += blockDim.x) {
    const int b = t / SO, u = t - b * SO;
    const int x = u % OX, y = (u / OX) % OY, z = u / (OX * OY);
    const int o = DIR == 0 ? x : (DIR == 1 ? y : z);
    const int base = b * SI + (DIR == 0 ? 0 : x) + (DIR == 1 ? 0 : y) * EX + (DIR == 2 ? 0 : z) * EX * EY;
    R acc = R(0);
#pragma unroll
    for (int m = 0; m < EIN; ++m) acc += (TR ? A[m * lda + o] : A[o * lda + m]) * in[base + m * SIN];
    out[t] = acc;
  }
}
template <int N, int NO, bool TR, typename R>
__device__ __forceinline__ void sweep3b(const R* A, int lda, const R* in, R* t0, R* t1, R* out, int ntens) {
  sweepb<N, N, N, 0, NO, TR>(A, lda, in, t0, ntens);
  __syncthreads();
  sweepb<NO, N, N, 1, NO, TR>(A, lda, t0, t1, ntens);
  __syncthreads();
  sweepb<NO, NO, N, 2, NO, TR>(A, lda, t1, out, ntens);
  __syncthreads();
}
template <int N, bool TR, typename R>
__device__ __forceinline__ void sweep_dirb(int dir, const R* A, const R* in, R* out, int ntens) {
  if (dir == 0) sweepb<N, N, N, 0, N, TR>(A, N, in, out, ntens);
  else if (dir == 1) sweepb<N, N, N, 1, N, TR>(A, N, in, out, ntens);
  else sweepb<N, N, N, 2, N, TR>(A, N, in, out, ntens);
}

// three sweeps with the same matrix (N -> NO per direction); tmp: two buffers of N^3
template <int N, int NO, bool TR, typename R>
__device__ __forceinline__ void sweep3(const R* A, int lda, const R* in, R* t0, R* t1, R* out) {
  sweep<N, N, N, 0, NO, TR>(A, lda, in, t0);
  __syncthreads();
  sweep<NO, N, N, 1, NO, TR>(A, lda, t0, t1);
  __syncthreads();
  sweep<NO, NO, N, 2, NO, TR>(A, lda, t1, out);
  __syncthreads();
}

// single sweep along a runtime direction (n^3 -> n^3)
template <int N, bool TR, typename R>
__device__ __forceinline__ void sweep_dir(int dir, const R* A, const R* in, R* out) {
  if (dir == 0) sweep<N, N, N, 0, N, TR>(A, N, in, out);
  else if (dir == 1) sweep<N, N, N, 1, N, TR>(A, N, in, out);
  else sweep<N, N, N, 2, N, TR>(A, N, in, out);
}

__device__ __forceinline__ void face_dirs(int d, int* t1, int* t2) {
  *t1 = d == 0 ? 1 : 0;
  *t2 = d == 2 ? 1 : 2;
}

// cell index of face point (a, b) (a along t1 < t2) of face (d, s) in an n^3 tensor
__device__ __forceinline__ int fnode(int d, int s, int a, int b, int n) {
  int i[3];
  int t1, t2;
  face_dirs(d, &t1, &t2);
  i[d] = s ? n - 1 : 0;
  i[t1] = a;
  i[t2] = b;
  return (i[2] * n + i[1]) * n + i[0];
}

// boundary-face number of the boundary face (e, f) (see LevelGeom)
__device__ __forceinline__ int bface_index(const LevelGeom& g, int e, int f) {
  if (g.nbr) return (-1 - g.nbr[e * 6 + f]) >> 3;
  const int ijk[3] = {e % g.nx, (e / g.nx) % g.ny, e / (g.nx * g.ny)};
  const int dims[3] = {g.nx, g.ny, g.nz};
  const int side[3] = {g.ny * g.nz, g.nx * g.nz, g.nx * g.ny};
  int off = 0;
  for (int s = 0; s < f; ++s) off += side[s >> 1];
  const int d = f >> 1;
  int t1, t2;
  face_dirs(d, &t1, &t2);
  return off + ijk[t2] * dims[t1] + ijk[t1];
}

// cell and face of boundary face b (inverse of bface_index)
__device__ __forceinline__ void bface_cell(const LevelGeom& g, int b, int* e, int* f) {
  if (g.bface) {
    const int v = g.bface[b];
    *e = v / 6;
    *f = v % 6;
    return;
  }
  int bf = b, ff = 0;
  const int side[3] = {g.ny * g.nz, g.nx * g.nz, g.nx * g.ny};
  while (bf >= side[ff >> 1]) {
    bf -= side[ff >> 1];
    ++ff;
  }
  const int d = ff >> 1, s = ff & 1;
  int t1, t2;
  face_dirs(d, &t1, &t2);
  const int dims[3] = {g.nx, g.ny, g.nz};
  int ijk[3];
  ijk[d] = s ? dims[d] - 1 : 0;
  ijk[t1] = bf % dims[t1];
  ijk[t2] = bf / dims[t1];
  *e = (ijk[2] * g.ny + ijk[1]) * g.nx + ijk[0];
  *f = ff;
}

// Wall velocity on the Dirichlet boundary faces: a constant vector per boundary
// id (g[6] for faces against removed cells), or, with pts != nullptr, values at
// the n^2 Gauss points of every boundary face, [nbf][n^2][3] (face point
// a + n b over the face's tangential directions t1 < t2).
struct Wall {
  double g[7][3];
  const double* pts;
};
__device__ __forceinline__ double wall_val(const Wall& w, const LevelGeom& g, int e, int f, int p, int c, int n2) {
  if (w.pts) return w.pts[((size_t)bface_index(g, e, f) * n2 + p) * 3 + c];
  return w.g[boundary_id(g, e, f)][c];
}

// load the split tables into shared memory (in the arithmetic type R of the kernel)
template <typename R>
struct STabSmT {
  R S[kMaxN * kMaxN], DS[kMaxN * kMaxN], Dg[kMaxN * kMaxN], Sp[kMaxN * kMaxN], DSp[kMaxN * kMaxN];
  R dS[2][kMaxN], lg[2][kMaxN], dlg[2][kMaxN], gw[kMaxN];
};
using STabSm = STabSmT<double>;
template <typename R>
__device__ __forceinline__ void load_tab(const SplitTab& t, STabSmT<R>& s) {
  for (int i = threadIdx.x; i < kMaxN * kMaxN; i += blockDim.x) {
    s.S[i] = t.S[i];
    s.DS[i] = t.DS[i];
    s.Dg[i] = t.Dg[i];
    s.Sp[i] = t.Sp[i];
    s.DSp[i] = t.DSp[i];
  }
  for (int i = threadIdx.x; i < kMaxN; i += blockDim.x) {
    s.dS[0][i] = t.dS0[i];
    s.dS[1][i] = t.dS1[i];
    s.lg[0][i] = t.lg0[i];
    s.lg[1][i] = t.lg1[i];
    s.dlg[0][i] = t.dlg0[i];
    s.dlg[1][i] = t.dlg1[i];
    s.gw[i] = t.gw[i];
  }
}

__device__ __forceinline__ double cell_weight(const STabSm& t, int q, int n, double detJ) {
  return t.gw[q % n] * t.gw[(q / n) % n] * t.gw[q / (n * n)] * detJ;
}

// trace on face (d, s) of a field F given at the n^3 Gauss points, with the 1D
// vector L over the normal index (values lg or derivatives dlg at 0 / 1)
template <int N, typename R>
__device__ __forceinline__ void trace(const R* F, const R* L, int d, R* out) {
  int t1, t2;
  face_dirs(d, &t1, &t2);
  const int str[3] = {1, N, N * N};
  for (int p = threadIdx.x; p < N * N; p += blockDim.x) {
    const int a = p % N, b = p / N;
    const int base = a * str[t1] + b * str[t2];
    R acc = R(0);
#pragma unroll
    for (int q = 0; q < N; ++q) acc += L[q] * F[base + q * str[d]];
    out[p] = acc;
  }
}

}  // namespace sweeps

// device copy of the wall data of the form launchers (split.cu)
sweeps::Wall make_wall(const WallArg& a);
}  // namespace sipg
