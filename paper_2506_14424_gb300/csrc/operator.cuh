// Matrix-free, sum-factorised SIPG operator kernels (element-centric, fused
// cell + face terms).
//
// Viscous operator, Eq. (viscous_term_weak) of the paper with the SIPG fluxes
// of Sec. 5.2 (u^dag = {{u}}, tau_1^dag = {{nu grad u}} - tau [[u]],
// tau_2^dag = (tau_1^dag)^T), summed over the faces of one cell:
//   cell:   (grad v, 2 nu eps(u))_e  [+ m (v, u)_e, Eq. viscous_step_weak]
//   face:   - (grad v : nu^- sym([u] (x) n))
//           - v . ( (A + A^T) n - tau ([u] + n ([u].n)) ),
//           A = (nu^- grad u^- + nu^+ grad u^+)/2,  [u] = u^- - u^+
//   Dirichlet wall: mirror u^+ = -u^-, grad u^+ = grad u^-, nu^+ = nu^-
//   Neumann wall:   no term (homogeneous flux data)
// Poisson operator, Eq. (pressure_step_weak) with the standard SIPG sign of
// the penalty (the printed "+ tau [[p]]" is read as a sign typo):
//   cell:   (grad q, grad p)_e
//   face:   - grad q . n [p]/2 - q ( {{grad p}}.n - tau [p] )
// Penalty tau = C_IP (k+1)^2 max(Lambda^-, Lambda^+) nubar(nu^-, nu^+)
// ("according to Hillewaert 2013", formula not printed; nubar = 1 for Poisson).
//
// Design: each CTA owns CPB consecutive cells and writes only their rows of y,
// so there are no atomics and the result is deterministic. Per cell:
//   1. stage x (own cell) in shared memory (contiguous, coalesced),
//   2. interpolate nodes -> Gauss points (3 sweeps), collocation gradient
//      (3 sweeps), quadrature-point flux, transposed sweeps back (6 sweeps),
//   3. per face: own trace and normal derivative from the staged nodes,
//      neighbour trace and normal derivative straight from global memory
//      (L2-resident), 2D interpolation to the face Gauss points, flux,
//      transposed 2D sweeps, scatter onto the cell's nodes,
//   4. store y once.
// All 1D contractions are "sweeps" over shared-memory tensors executed
// cooperatively by the CTA's threads.
#pragma once
#include "common.cuh"
#include "ff.cuh"

namespace sipg {

template <typename T>
__device__ __forceinline__ T nubar_of(int mode, T a, T b) {
  if (mode == 1) return T(0.5f) * (a + b);
  if (mode == 2) return T(2) * a * b / (a + b);
  return a > b ? a : b;
}

// out[t][.. o ..] (+)= sum_j M(o, j) in[t][.. j ..] along direction DIR of
// N^3 tensors (x fastest); M(o, j) = M[o*N + j], or M[j*N + o] if TR.
template <int N, int DIR, bool TR, bool ACC, typename T>
__device__ __forceinline__ void sweep3(const T* __restrict__ in, T* __restrict__ out,
                                       const T* __restrict__ M, int ntens) {
  constexpr int N3 = N * N * N;
  constexpr int STR = DIR == 0 ? 1 : (DIR == 1 ? N : N * N);
  for (int idx = threadIdx.x; idx < ntens * N3; idx += blockDim.x) {
    const int t = idx / N3, r = idx - t * N3;
    const int o = (r / STR) % N;
    const T* base = in + t * N3 + (r - o * STR);
    Acc<T> acc;
#pragma unroll
    for (int j = 0; j < N; ++j) acc.add(TR ? M[j * N + o] : M[o * N + j], base[j * STR]);
    out[idx] = ACC ? out[idx] + acc.get() : acc.get();
  }
}

// Same on N^2 face tensors (a fastest): DIR 0 along a, 1 along b.
template <int N, int DIR, bool TR, bool ACC, typename T>
__device__ __forceinline__ void sweep2(const T* __restrict__ in, T* __restrict__ out,
                                       const T* __restrict__ M, int ntens) {
  constexpr int N2 = N * N;
  constexpr int STR = DIR == 0 ? 1 : N;
  for (int idx = threadIdx.x; idx < ntens * N2; idx += blockDim.x) {
    const int t = idx / N2, r = idx - t * N2;
    const int o = (r / STR) % N;
    const T* base = in + t * N2 + (r - o * STR);
    Acc<T> acc;
#pragma unroll
    for (int j = 0; j < N; ++j) acc.add(TR ? M[j * N + o] : M[o * N + j], base[j * STR]);
    out[idx] = ACC ? out[idx] + acc.get() : acc.get();
  }
}

// Offset inside an N^3 cell tensor of the node with index `layer` along d and
// (a, b) along the tangential directions t1 < t2 of d.
template <int N>
__device__ __forceinline__ int face_node(int d, int layer, int a, int b) {
  constexpr int N2 = N * N;
  if (d == 0) return layer + a * N + b * N2;        // t1 = y, t2 = z
  if (d == 1) return a + layer * N + b * N2;        // t1 = x, t2 = z
  return a + b * N + layer * N2;                    // t1 = x, t2 = y
}
template <int N>
__device__ __forceinline__ int dir_stride(int d) { return d == 0 ? 1 : (d == 1 ? N : N * N); }

// Cells per CTA and threads per CTA of the operator kernels.
template <int N> struct OpCfg {
  static constexpr int CPB = N == 2 ? 32 : (N == 3 ? 8 : (N == 4 ? 4 : 2));
  static constexpr int NT = 256;
};

// Shared-memory footprint (in elements of T) of apply_kernel.
template <int N, int NC>
__host__ __device__ constexpr int op_smem_elems() {
  return 3 * N * N + 4 * N + OpCfg<N>::CPB * (5 * NC * N * N * N + 16 * NC * N * N);
}

template <int N, typename T>
__device__ __forceinline__ void load_tables(const Tab& tab, T* S, T* Dg, T* dS0, T* dS1, T* gw) {
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    S[i] = from_double<T>(tab.S[i]);
    Dg[i] = from_double<T>(tab.Dg[i]);
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    dS0[i] = from_double<T>(tab.dS0[i]);
    dS1[i] = from_double<T>(tab.dS1[i]);
    gw[i] = from_double<T>(tab.gw[i]);
  }
}

// y = (m M + A) x on the cells [blockIdx.x*CPB, ...) of a level.
// NC = 3: viscous operator (nu_cell [C][N^3], nu_face [C][6][N^2]);
// NC = 1: Poisson operator (nu pointers unused).
// TS is the storage type of x, y and nu; T the arithmetic type (double,
// float, or ff = float-float with double storage).
template <int N, int NC, typename TS, typename T>
__global__ void __launch_bounds__(OpCfg<N>::NT)
apply_kernel(LevelGeom g, Tab tab, const TS* __restrict__ x, TS* __restrict__ y,
             const TS* __restrict__ nu_cell, const TS* __restrict__ nu_face, double mass_d, int64_t batch_stride) {
  const T mass = from_double<T>(mass_d);
  constexpr int N2 = N * N, N3 = N * N * N, CPB = OpCfg<N>::CPB;
  // blockIdx.y selects one of several vectors applied in the same launch
  x += (int64_t)blockIdx.y * batch_stride;
  y += (int64_t)blockIdx.y * batch_stride;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* S = sm;
  T* Dg = S + N2;
  T* dS0 = Dg + N2;
  T* dS1 = dS0 + N;
  T* gw = dS1 + N;
  T* buf = sm + 3 * N2 + 4 * N;
  T* Xs = buf;
  T* U = Xs + CPB * NC * N3;
  T* B1 = U + CPB * NC * N3;
  T* B2 = B1 + CPB * NC * N3;
  T* B3 = B2 + CPB * NC * N3;
  T* F = B3 + CPB * NC * N3;  // 16 face slots of CPB*NC*N2
  const int FS = CPB * NC * N2;
  T *sV = F, *sN = F + FS, *pV = F + 2 * FS, *pN = F + 3 * FS;
  T *T1 = F + 4 * FS, *T2 = F + 5 * FS, *T3 = F + 6 * FS, *T4 = F + 7 * FS;
  T *gV = F + 8 * FS, *gN = F + 9 * FS, *gT1 = F + 10 * FS, *gT2 = F + 11 * FS;
  T *gVp = F + 12 * FS, *gNp = F + 13 * FS, *gT1p = F + 14 * FS, *gT2p = F + 15 * FS;

  load_tables<N>(tab, S, Dg, dS0, dS1, gw);
  const int cell0 = blockIdx.x * CPB;
  const int ncell = min(CPB, g.ncells - cell0);
  const int nt = ncell * NC;
  const size_t base0 = (size_t)cell0 * NC * N3;
  for (int i = threadIdx.x; i < nt * N3; i += blockDim.x) Xs[i] = load_as<T>(x[base0 + i]);
  __syncthreads();

  // ---- cell term: values at Gauss points, then the collocation gradient
  sweep3<N, 0, false, false>(Xs, B1, S, nt);
  __syncthreads();
  sweep3<N, 1, false, false>(B1, B2, S, nt);
  __syncthreads();
  sweep3<N, 2, false, false>(B2, U, S, nt);
  __syncthreads();
  sweep3<N, 0, false, false>(U, B1, Dg, nt);
  sweep3<N, 1, false, false>(U, B2, Dg, nt);
  sweep3<N, 2, false, false>(U, B3, Dg, nt);
  __syncthreads();
  const T ih[3] = {from_double<T>(g.ih[0]), from_double<T>(g.ih[1]), from_double<T>(g.ih[2])};
  const T detJ = from_double<T>(g.h[0] * g.h[1] * g.h[2]);
  for (int i = threadIdx.x; i < ncell * N3; i += blockDim.x) {
    const int c = i / N3, q = i - c * N3;
    const int qx = q % N, qy = (q / N) % N, qz = q / N2;
    const T W = gw[qx] * gw[qy] * gw[qz] * detJ;
    T* Bl[3] = {B1, B2, B3};
    if constexpr (NC == 3) {
      T G[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) G[k][l] = Bl[l][(c * 3 + k) * N3 + q] * ih[l];
      const T nu2W = T(2) * load_as<T>(nu_cell[(size_t)(cell0 + c) * N3 + q]) * W;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int l = 0; l < 3; ++l)
          Bl[l][(c * 3 + k) * N3 + q] = nu2W * T(0.5f) * (G[k][l] + G[l][k]) * ih[l];
        U[(c * 3 + k) * N3 + q] *= mass * W;
      }
    } else {
#pragma unroll
      for (int l = 0; l < 3; ++l) Bl[l][c * N3 + q] = Bl[l][c * N3 + q] * ih[l] * W * ih[l];
      U[c * N3 + q] *= mass * W;
    }
  }
  __syncthreads();
  sweep3<N, 0, true, true>(B1, U, Dg, nt);
  sweep3<N, 1, true, true>(B2, U, Dg, nt);
  sweep3<N, 2, true, true>(B3, U, Dg, nt);
  __syncthreads();
  sweep3<N, 2, true, false>(U, B1, S, nt);
  __syncthreads();
  sweep3<N, 1, true, false>(B1, B2, S, nt);
  __syncthreads();
  sweep3<N, 0, true, false>(B2, B3, S, nt);  // B3 = cell contribution to y
  __syncthreads();

  // ---- face terms, one face direction/side at a time
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    const int fo = f ^ 1;
    const int layer = s ? N - 1 : 0, layer_nb = s ? 0 : N - 1;
    const T* dS = s ? dS1 : dS0;
    const T* dSn = s ? dS0 : dS1;
    const int std_ = dir_stride<N>(d);
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    // traces and normal derivatives at the face Gauss-Lobatto nodes
    for (int i = threadIdx.x; i < nt * N2; i += blockDim.x) {
      const int t = i / N2, p = i - t * N2;
      const int a = p % N, b = p / N;
      const int c = t / NC, comp = t - c * NC;
      const int e = cell0 + c;
      const int off0 = face_node<N>(d, 0, a, b);
      const T* xs = Xs + t * N3 + off0;
      Acc<T> dn;
#pragma unroll
      for (int j = 0; j < N; ++j) dn.add(dS[j], xs[j * std_]);
      sV[i] = xs[layer * std_];
      sN[i] = dn.get();
      const int nb = cell_neighbor(g, e, f);
      if (nb >= 0) {
        const TS* xn = x + ((size_t)nb * NC + comp) * N3 + off0;
        Acc<T> dnn;
#pragma unroll
        for (int j = 0; j < N; ++j) dnn.add(dSn[j], load_as<T>(xn[j * std_]));
        pV[i] = load_as<T>(xn[layer_nb * std_]);
        pN[i] = dnn.get();
      } else {
        pV[i] = T(0);
        pN[i] = T(0);
      }
    }
    __syncthreads();
    sweep2<N, 0, false, false>(sV, T1, S, nt);
    sweep2<N, 0, false, false>(sN, T2, S, nt);
    sweep2<N, 0, false, false>(pV, T3, S, nt);
    sweep2<N, 0, false, false>(pN, T4, S, nt);
    __syncthreads();
    sweep2<N, 1, false, false>(T1, gV, S, nt);
    sweep2<N, 1, false, false>(T2, gN, S, nt);
    sweep2<N, 1, false, false>(T3, gVp, S, nt);
    sweep2<N, 1, false, false>(T4, gNp, S, nt);
    __syncthreads();
    sweep2<N, 0, false, false>(gV, gT1, Dg, nt);
    sweep2<N, 1, false, false>(gV, gT2, Dg, nt);
    sweep2<N, 0, false, false>(gVp, gT1p, Dg, nt);
    sweep2<N, 1, false, false>(gVp, gT2p, Dg, nt);
    __syncthreads();
    // numerical flux at the face quadrature points
    const T nsign = s ? T(1) : T(-1);
    const T ihd = ih[d], iht1 = ih[t1], iht2 = ih[t2];
    const T area = from_double<T>(g.h[t1] * g.h[t2]);
    for (int i = threadIdx.x; i < ncell * N2; i += blockDim.x) {
      const int c = i / N2, p = i - c * N2;
      const int a = p % N, b = p / N;
      const int e = cell0 + c;
      const int nb = cell_neighbor(g, e, f);
      const bool neumann = nb < 0 && g.bc[f] == 1;
      if (neumann) {
        for (int k = 0; k < NC; ++k) {
          const int j = (c * NC + k) * N2 + p;
          gV[j] = T(0); gN[j] = T(0); gT1[j] = T(0); gT2[j] = T(0);
        }
        continue;
      }
      const T W = gw[a] * gw[b] * area;
      const double lam_md = penalty_lambda(g, e);
      const double lam_pd = nb >= 0 ? penalty_lambda(g, nb) : lam_md;
      // C_IP (k+1)^2 max(Lambda-, Lambda+): geometry only, formed in FP64 once
      const T pen = from_double<T>(g.cip * double(N * N) * (lam_md > lam_pd ? lam_md : lam_pd));
      if constexpr (NC == 3) {
        const T num = load_as<T>(nu_face[((size_t)e * 6 + f) * N2 + p]);
        const T nup = nb >= 0 ? load_as<T>(nu_face[((size_t)nb * 6 + fo) * N2 + p]) : num;
        const T tau = pen * nubar_of<T>(g.face_nu, num, nup);
        T um[3], up[3], Gm[3][3], Gp[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int j = (c * 3 + k) * N2 + p;
          um[k] = gV[j];
          Gm[k][d] = gN[j] * ihd;
          Gm[k][t1] = gT1[j] * iht1;
          Gm[k][t2] = gT2[j] * iht2;
          if (nb >= 0) {
            up[k] = gVp[j];
            Gp[k][d] = gNp[j] * ihd;
            Gp[k][t1] = gT1p[j] * iht1;
            Gp[k][t2] = gT2p[j] * iht2;
          }
        }
        if (nb < 0) {  // Dirichlet mirror
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            up[k] = -um[k];
#pragma unroll
            for (int l = 0; l < 3; ++l) Gp[k][l] = Gm[k][l];
          }
        }
        T jmp[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) jmp[k] = um[k] - up[k];
        const T jn = jmp[d] * nsign;
        // (A + A^T) n with A = (nu^- G^- + nu^+ G^+)/2 and n = nsign e_d
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const T Akd = T(0.5f) * (num * Gm[k][d] + nup * Gp[k][d]);
          const T Adk = T(0.5f) * (num * Gm[d][k] + nup * Gp[d][k]);
          const T nk = k == d ? nsign : T(0);
          const T P = -((Akd + Adk) * nsign - tau * (jmp[k] + nk * jn));
          // test-gradient coefficient Q = -nu^- sym(jump (x) n)
          // Q[k][l] = -nu^- (jmp_k n_l + n_k jmp_l) / 2
          const T Qkd = -num * T(0.5f) * (jmp[k] * nsign + nk * jmp[d]);
          const T Qkt1 = -num * T(0.5f) * (k == d ? nsign * jmp[t1] : T(0));
          const T Qkt2 = -num * T(0.5f) * (k == d ? nsign * jmp[t2] : T(0));
          const int j = (c * 3 + k) * N2 + p;
          gV[j] = W * P;
          gN[j] = W * Qkd * ihd;
          gT1[j] = W * Qkt1 * iht1;
          gT2[j] = W * Qkt2 * iht2;
        }
      } else {
        const T tau = pen;
        const int j = c * N2 + p;
        const T pm = gV[j];
        const T dnm = gN[j] * ihd;
        T pp, dnp;
        if (nb >= 0) {
          pp = gVp[j];
          dnp = gNp[j] * ihd;
        } else {
          pp = -pm;
          dnp = dnm;
        }
        const T jmp = pm - pp;
        // -grad q . n jump/2 - q ({{dp/dx_d}} n_d - tau jump)
        gV[j] = -W * (T(0.5f) * (dnm + dnp) * nsign - tau * jmp);
        gN[j] = -W * T(0.5f) * jmp * nsign * ihd;
        gT1[j] = T(0);
        gT2[j] = T(0);
      }
    }
    __syncthreads();
    sweep2<N, 0, true, true>(gT1, gV, Dg, nt);
    sweep2<N, 1, true, true>(gT2, gV, Dg, nt);
    __syncthreads();
    sweep2<N, 1, true, false>(gV, T1, S, nt);
    sweep2<N, 1, true, false>(gN, T2, S, nt);
    __syncthreads();
    sweep2<N, 0, true, false>(T1, sV, S, nt);
    sweep2<N, 0, true, false>(T2, sN, S, nt);
    __syncthreads();
    for (int i = threadIdx.x; i < nt * N3; i += blockDim.x) {
      const int t = i / N3, r = i - t * N3;
      const int ix = r % N, iy = (r / N) % N, iz = r / N2;
      const int id = d == 0 ? ix : (d == 1 ? iy : iz);
      const int a = d == 0 ? iy : ix;
      const int b = d == 2 ? iy : iz;
      const int fp = t * N2 + a + N * b;
      T v = dS[id] * sN[fp];
      if (id == layer) v += sV[fp];
      B3[i] += v;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nt * N3; i += blockDim.x) y[base0 + i] = store_as<TS>(B3[i]);
}

}  // namespace sipg
