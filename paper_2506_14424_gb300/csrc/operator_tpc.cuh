// Register-tiled FP32 SIPG operator kernel for low degrees (n = k+1 <= 4).
//
// The same operator as operator.cuh (Eq. viscous_term_weak with the SIPG
// fluxes of Sec. 5.2, or the Poisson form of Eq. pressure_step_weak, plus the
// optional mass term of Eq. viscous_step_weak), mapped differently: one
// thread owns one (cell, component) pair and keeps the cell's n^3 values of
// that component in registers, so every 1D sum-factorisation sweep is a chain
// of register FMAs with the 1D matrices as constant-bank operands and no
// shared-memory traffic. Threads exchange data only where the components
// couple:
//   * cell term (viscous): the 3 x 3 velocity gradient at the Gauss points
//     (each thread publishes its component's three gradient tiles, reads the
//     transposed entries), for 2 nu eps(u);
//   * faces (viscous): the jump of each component and the tangential
//     derivatives of the normal component at the face Gauss points.
// A warp holds CW whole cells (10 cells x 3 components, lanes 30, 31 idle; or
// 32 cells of the scalar Poisson operator) and a CTA is one warp, so every
// exchange is warp-local (__syncwarp) and the kernel has no CTA barrier.
// Neighbour traces are read from global memory (L2) as float4 rows of the
// neighbour's tile. Each thread writes only its own cell's rows of y: no
// atomics, deterministic.
#pragma once
#include "common.cuh"
#include "ff.cuh"
#include "operator.cuh"

namespace sipg {

// 1D tables in FP32 (kernel parameter: compile-time indices become
// constant-bank operands). Same definitions as Tab.
struct TpcTab {
  float S[kMaxN * kMaxN];
  float Dg[kMaxN * kMaxN];
  float dS0[kMaxN], dS1[kMaxN], gw[kMaxN];
};

template <int NC>
struct TpcCfg {
  static constexpr int CW = NC == 3 ? 10 : 32;  // cells per warp
};

// Strides of the warp's shared exchange regions, padded so that the lanes of a
// warp hit distinct banks (at most 2-way conflicts; found by enumerating the
// access patterns below for 10 cells x 3 components and 32 cells):
//   gradient tiles  G[cw*GC + (dir*3 + comp)*GT + q]   (cell term, viscous)
//   face data       E[(cw*3 + comp)*EC + slot*ES + p]  (faces, viscous; 5 slots)
//   scalar values   U[cw*UC + q]                       (cell term, Poisson)
template <int N> struct TpcPad;
template <> struct TpcPad<2> { static constexpr int GT = 8, GC = 73, ES = 4, EC = 21, UC = 9; };
template <> struct TpcPad<3> { static constexpr int GT = 27, GC = 243, ES = 9, EC = 45, UC = 27; };
template <> struct TpcPad<4> { static constexpr int GT = 65, GC = 585, ES = 16, EC = 81, UC = 65; };

// Shared floats per warp.
template <int N, int NC>
__host__ __device__ constexpr int tpc_smem_floats() {
  return NC == 3 ? (TpcPad<N>::GC * TpcCfg<NC>::CW > 3 * TpcPad<N>::EC * TpcCfg<NC>::CW
                        ? TpcPad<N>::GC * TpcCfg<NC>::CW
                        : 3 * TpcPad<N>::EC * TpcCfg<NC>::CW)
                 : TpcPad<N>::UC * TpcCfg<NC>::CW;
}

// ---- register sweeps on an N^3 tile t[(iz*N + iy)*N + ix]
// t_line <- M t_line (TR: M^T) along direction DIR, in place
template <int N, int DIR, bool TR>
__device__ __forceinline__ void rsweep3(float (&t)[N * N * N], const float* M) {
  constexpr int N2 = N * N;
  constexpr int STR = DIR == 0 ? 1 : (DIR == 1 ? N : N2);
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int b = 0; b < N; ++b) {
      const int off = DIR == 0 ? (a * N + b * N2) : (DIR == 1 ? (a + b * N2) : (a + b * N));
      float v[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = t[off + j * STR];
#pragma unroll
      for (int o = 0; o < N; ++o) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) s = fmaf(TR ? M[j * N + o] : M[o * N + j], v[j], s);
        t[off + o * STR] = s;
      }
    }
}
// the same on an N^2 face tensor f[b*N + a] (DIR 0: along a, 1: along b)
template <int N, int DIR, bool TR>
__device__ __forceinline__ void rsweep2(float (&f)[N * N], const float* M) {
  constexpr int STR = DIR == 0 ? 1 : N;
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const int off = DIR == 0 ? r * N : r;
    float v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = f[off + j * STR];
#pragma unroll
    for (int o = 0; o < N; ++o) {
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < N; ++j) s = fmaf(TR ? M[j * N + o] : M[o * N + j], v[j], s);
      f[off + o * STR] = s;
    }
  }
}
// out = M f along DIR (f unchanged)
template <int N, int DIR>
__device__ __forceinline__ void rderiv2(const float (&f)[N * N], float (&out)[N * N], const float* M) {
  constexpr int STR = DIR == 0 ? 1 : N;
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const int off = DIR == 0 ? r * N : r;
#pragma unroll
    for (int o = 0; o < N; ++o) {
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < N; ++j) s = fmaf(M[o * N + j], f[off + j * STR], s);
      out[off + o * STR] = s;
    }
  }
}

// Load an N^3 FP32 tile (float4 rows where the tile size allows).
template <int N>
__device__ __forceinline__ void load_tile(const float* __restrict__ src, float (&t)[N * N * N]) {
  constexpr int N3 = N * N * N;
  if constexpr (N3 % 4 == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int i = 0; i < N3 / 4; ++i) {
      const float4 v = __ldg(s4 + i);
      t[4 * i] = v.x; t[4 * i + 1] = v.y; t[4 * i + 2] = v.z; t[4 * i + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N3; ++i) t[i] = __ldg(src + i);
  }
}

// One row (fixed iy, iz; ix = 0..N-1) of an N^3 FP32 tile in global memory.
template <int N>
__device__ __forceinline__ void load_row(const float* __restrict__ src, float (&r)[N]) {
  if constexpr (N == 4) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(src));
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
  } else if constexpr (N == 2) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(src));
    r[0] = v.x; r[1] = v.y;
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) r[i] = __ldg(src + i);
  }
}

// Trace (layer `layer` along D) and normal derivative dS . line at the face
// nodes (a, b) of a tile in global memory, a along the lower tangential
// direction t1, b along t2 (the node order of face_node in operator.cuh),
// streamed row by row.
template <int N, int D>
__device__ __forceinline__ void face_trace(const float* __restrict__ src, bool last, const float (&dS)[N],
                                           float (&tr)[N * N], float (&nd)[N * N]) {
  constexpr int N2 = N * N;
  if constexpr (D == 0) {  // lines along x are rows (a = iy, b = iz)
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int a = 0; a < N; ++a) {
        float r[N];
        load_row<N>(src + (b * N + a) * N, r);
        float sd = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) sd = fmaf(dS[j], r[j], sd);
        nd[b * N + a] = sd;
        tr[b * N + a] = last ? r[N - 1] : r[0];
      }
  } else {  // D = 1: a = ix, b = iz, rows (iy = j, iz = b); D = 2: a = ix, b = iy, rows (iy = b, iz = j)
#pragma unroll
    for (int p = 0; p < N2; ++p) nd[p] = 0.f;
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int j = 0; j < N; ++j) {
        float r[N];
        load_row<N>(src + (D == 1 ? (b * N2 + j * N) : (j * N2 + b * N)), r);
#pragma unroll
        for (int a = 0; a < N; ++a) {
          nd[b * N + a] = fmaf(dS[j], r[a], nd[b * N + a]);
          if (j == 0 && !last) tr[b * N + a] = r[a];
          if (j == N - 1 && last) tr[b * N + a] = r[a];
        }
      }
  }
}

// Lambda_e = sum_f w_f / h_{f/2} (w = 1/2 interior, 1 boundary) in FP32
template <bool TOPO>
__device__ __forceinline__ float lambda_f(const LevelGeom& g, int e, const int* ijk, const float* ihf) {
  float lam = 0.f;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    bool bnd;
    if (TOPO) {
      bnd = g.nbr[e * 6 + f] < 0;
    } else {
      const int d = f >> 1;
      const int dims = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
      bnd = (f & 1) ? ijk[d] == dims - 1 : ijk[d] == 0;
    }
    lam += (bnd ? 1.0f : 0.5f) * ihf[f >> 1];
  }
  return lam;
}

// Face terms of direction D (both sides) added to the nodal accumulator t.
template <int N, int NC, bool TOPO, int D>
__device__ __forceinline__ void tpc_faces(const LevelGeom& g, const TpcTab& tb, const float* __restrict__ x,
                                          const float* __restrict__ xe, const float* __restrict__ nu_face, int e,
                                          int kk, int cw, bool active, const int* ijk, const float* ihf, float lam_e,
                                          const LevelConsts<float>& lc, float (&t)[N * N * N], float* tsm) {
  constexpr int N2 = N * N, N3 = N2 * N;
  (void)N3;
  const int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
  const float ihd = ihf[D], iht1 = ihf[T1], iht2 = ihf[T2];
  const float area = lc.area[D];
#pragma unroll 1
  for (int s = 0; s < 2; ++s) {
    const int f = 2 * D + s;
    int nb;
    if (TOPO) {
      const int v = g.nbr[e * 6 + f];
      nb = v >= 0 ? v : -1;
    } else {
      const int dims = D == 0 ? g.nx : (D == 1 ? g.ny : g.nz);
      const bool bnd = s ? ijk[D] == dims - 1 : ijk[D] == 0;
      const int step = D == 0 ? 1 : (D == 1 ? g.nx : g.nx * g.ny);
      nb = bnd ? -1 : e + (s ? step : -step);
    }
    const bool inner = nb >= 0;
    const int bcf = TOPO ? face_bc_t<TOPO>(g, e, f) : (s ? g.bc[2 * D + 1] : g.bc[2 * D]);
    const bool neumann = !inner && bcf == 1;
    // normal-derivative rows of the own side and of the neighbour's side (registers:
    // the side index is a loop variable)
    float dso[N], dsn[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      dso[j] = s ? tb.dS1[j] : tb.dS0[j];
      dsn[j] = s ? tb.dS0[j] : tb.dS1[j];
    }
    // own and neighbour traces / normal derivatives at the face nodes
    float tm[N2], nm[N2], tp[N2], np[N2];
    face_trace<N, D>(xe, s != 0, dso, tm, nm);
    if (inner) {
      face_trace<N, D>(x + ((size_t)nb * NC + kk) * N3, s == 0, dsn, tp, np);
    }
    // to the face Gauss points (a then b)
    rsweep2<N, 0, false>(tm, tb.S);
    rsweep2<N, 1, false>(tm, tb.S);
    rsweep2<N, 0, false>(nm, tb.S);
    rsweep2<N, 1, false>(nm, tb.S);
    if (inner) {
      rsweep2<N, 0, false>(tp, tb.S);
      rsweep2<N, 1, false>(tp, tb.S);
      rsweep2<N, 0, false>(np, tb.S);
      rsweep2<N, 1, false>(np, tb.S);
    } else {  // Dirichlet mirror u+ = -u-, grad u+ = grad u- (Neumann: unused)
#pragma unroll
      for (int p = 0; p < N2; ++p) {
        tp[p] = -tm[p];
        np[p] = nm[p];
      }
    }
    float pe;
    {
      float lam_n = lam_e;
      if (inner) {
        int nijk[3] = {ijk[0], ijk[1], ijk[2]};
        if (!TOPO) nijk[D] += s ? 1 : -1;
        lam_n = lambda_f<TOPO>(g, nb, nijk, ihf);
      }
      pe = lc.cipn2 * fmaxf(lam_e, lam_n);
    }
    const float nsign = s ? 1.f : -1.f;
    float gV[N2], gN[N2];
    if constexpr (NC == 3) {
      // publish the jump and the tangential derivatives (own, neighbour)
      constexpr int ES = TpcPad<N>::ES, EC = TpcPad<N>::EC;
      float* EX = tsm + (cw * 3 + kk) * EC;
      float d1[N2], d2[N2];
      rderiv2<N, 0>(tm, d1, tb.Dg);
      rderiv2<N, 1>(tm, d2, tb.Dg);
      if (active) {
#pragma unroll
        for (int p = 0; p < N2; ++p) {
          EX[p] = tm[p] - tp[p];
          EX[ES + p] = d1[p] * iht1;
          EX[2 * ES + p] = d2[p] * iht2;
        }
      }
      if (inner) {
        rderiv2<N, 0>(tp, d1, tb.Dg);
        rderiv2<N, 1>(tp, d2, tb.Dg);
      }
      if (active) {
#pragma unroll
        for (int p = 0; p < N2; ++p) {
          EX[3 * ES + p] = d1[p] * iht1;
          EX[4 * ES + p] = d2[p] * iht2;
        }
      }
      __syncwarp();
      const float* ED = tsm + (cw * 3 + D) * EC;     // the normal component's data
      const float* E1 = tsm + (cw * 3 + T1) * EC;
      const float* E2 = tsm + (cw * 3 + T2) * EC;
      const bool isD = kk == D;
      const int tsel = kk == T1 ? 1 : 2;                 // tangential direction of this component
      const float* nuf = nu_face + ((size_t)e * 6 + f) * N2;
      const float* nufp = nu_face + ((size_t)(inner ? nb : e) * 6 + (inner ? (f ^ 1) : f)) * N2;
      float gT1[N2], gT2[N2];
#pragma unroll
      for (int p = 0; p < N2; ++p) {
        const int a = p % N, b = p / N;
        const float W = tb.gw[a] * tb.gw[b] * area;
        const float num = __ldg(nuf + p);
        const float nup = __ldg(nufp + p);
        const float nb_ = g.face_nu == 1 ? 0.5f * (num + nup)
                                         : (g.face_nu == 2 ? 2.f * num * nup / (num + nup) : fmaxf(num, nup));
        const float tW = pe * nb_ * W;
        const float am = 0.5f * nsign * num * W, ap = 0.5f * nsign * nup * W, cq = -am;
        const float jmp = tm[p] - tp[p];
        if (isD) {
          gV[p] = 2.f * (tW * jmp - (am * nm[p] + ap * np[p]) * ihd);
          gN[p] = 2.f * cq * jmp * ihd;
          gT1[p] = cq * E1[p] * iht1;
          gT2[p] = cq * E2[p] * iht2;
        } else {
          const float tmk = ED[tsel * ES + p];
          const float tpk = inner ? ED[(tsel + 2) * ES + p] : tmk;
          gV[p] = tW * jmp - (am * (nm[p] * ihd + tmk) + ap * (np[p] * ihd + tpk));
          gN[p] = cq * jmp * ihd;
          gT1[p] = 0.f;
          gT2[p] = 0.f;
        }
      }
      __syncwarp();  // the next face reuses the exchange region
      // test side: V + Dg_a^T T1 + Dg_b^T T2, then S^T along b and a
#pragma unroll
      for (int r = 0; r < N; ++r)
#pragma unroll
        for (int o = 0; o < N; ++o) {
          float s1 = gV[r * N + o], s2 = 0.f;
#pragma unroll
          for (int j = 0; j < N; ++j) {
            s1 = fmaf(tb.Dg[j * N + o], gT1[r * N + j], s1);   // along a (row r = b)
            s2 = fmaf(tb.Dg[j * N + r], gT2[j * N + o], s2);   // along b (column o = a)
          }
          gV[r * N + o] = s1 + s2;
        }
    } else {
#pragma unroll
      for (int p = 0; p < N2; ++p) {
        const int a = p % N, b = p / N;
        const float W = tb.gw[a] * tb.gw[b] * area;
        const float dnm = nm[p] * ihd, dnp = np[p] * ihd;
        const float jmp = tm[p] - tp[p];
        gV[p] = -W * (0.5f * (dnm + dnp) * nsign - pe * jmp);
        gN[p] = -W * 0.5f * jmp * nsign * ihd;
      }
    }
    rsweep2<N, 1, true>(gV, tb.S);
    rsweep2<N, 0, true>(gV, tb.S);
    rsweep2<N, 1, true>(gN, tb.S);
    rsweep2<N, 0, true>(gN, tb.S);
    if (!neumann) {
      constexpr int STR = D == 0 ? 1 : (D == 1 ? N : N2);
#pragma unroll
      for (int b = 0; b < N; ++b)
#pragma unroll
        for (int a = 0; a < N; ++a) {
          const int base = D == 0 ? (a * N + b * N2) : (D == 1 ? (a + b * N2) : (a + b * N));
#pragma unroll
          for (int j = 0; j < N; ++j) t[base + j * STR] = fmaf(dso[j], gN[b * N + a], t[base + j * STR]);
          const float vlast = s ? gV[b * N + a] : 0.f;
          t[base] += gV[b * N + a] - vlast;
          t[base + (N - 1) * STR] += vlast;
        }
    }
  }
}

template <int N, int NC, bool TOPO>
__global__ void __launch_bounds__(32, 8)
apply_tpc_kernel(LevelGeom g, TpcTab tb, LevelConsts<float> lc, const float* __restrict__ x,
                 float* __restrict__ y, const float* __restrict__ nu_cell, const float* __restrict__ nu_face,
                 int64_t batch_stride) {
  constexpr int N2 = N * N, N3 = N2 * N, CW = TpcCfg<NC>::CW;
  extern __shared__ __align__(16) float tsm[];
  x += (int64_t)blockIdx.y * batch_stride;
  y += (int64_t)blockIdx.y * batch_stride;
  const int lane = threadIdx.x;
  const int k = NC == 3 ? lane / CW : 0;        // component
  const int cw = NC == 3 ? lane - k * CW : lane;  // cell within the warp
  const bool active = k < NC;                     // lanes 30, 31 of the viscous kernel idle
  const int cell_raw = blockIdx.x * CW + cw;
  const bool store = active && cell_raw < g.ncells;
  const int e = min(cell_raw, g.ncells - 1);
  const int kk = active ? k : 0;
  const float ihf[3] = {lc.ih[0], lc.ih[1], lc.ih[2]};
  const float detJ = lc.detJ;
  const float mass = lc.mass;
  int ijk[3] = {0, 0, 0};
  if (!TOPO) {
    ijk[0] = e % g.nx;
    ijk[1] = (e / g.nx) % g.ny;
    ijk[2] = e / (g.nx * g.ny);
  }
  const float* xe = x + ((size_t)e * NC + kk) * N3;

  // ------------------------------------------------------------- cell term
  float t[N3];
  load_tile<N>(xe, t);
  rsweep3<N, 0, false>(t, tb.S);
  rsweep3<N, 1, false>(t, tb.S);
  rsweep3<N, 2, false>(t, tb.S);  // t = u_k at the Gauss points
  if constexpr (NC == 3) {
    // publish the physical gradient tiles: G(dir l, comp k)[q] = d u_k / d x_l
    constexpr int GT = TpcPad<N>::GT, GC = TpcPad<N>::GC;
    float* G = tsm + cw * GC + kk * GT;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const int STR = l == 0 ? 1 : (l == 1 ? N : N2);
#pragma unroll
      for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
          const int off = l == 0 ? (a * N + b * N2) : (l == 1 ? (a + b * N2) : (a + b * N));
#pragma unroll
          for (int o = 0; o < N; ++o) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < N; ++j) s = fmaf(tb.Dg[o * N + j], t[off + j * STR], s);
            if (active) G[l * 3 * GT + off + o * STR] = s * ihf[l];
          }
        }
    }
    __syncwarp();
    // acc = mass W u, then + D_l^T F_kl with F_kl = nu W (G_kl + G_lk) / h_l
#pragma unroll
    for (int q = 0; q < N3; ++q) {
      const float W = tb.gw[q % N] * tb.gw[(q / N) % N] * tb.gw[q / N2] * detJ;
      t[q] *= mass * W;
    }
    const float* Gc = tsm + cw * GC;
    const float* nue = nu_cell + (size_t)e * N3;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const int STR = l == 0 ? 1 : (l == 1 ? N : N2);
#pragma unroll
      for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
          const int off = l == 0 ? (a * N + b * N2) : (l == 1 ? (a + b * N2) : (a + b * N));
          float F[N];
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const int q = off + j * STR;
            const float W = tb.gw[q % N] * tb.gw[(q / N) % N] * tb.gw[q / N2] * detJ;
            F[j] = __ldg(nue + q) * W * (Gc[(l * 3 + kk) * GT + q] + Gc[(kk * 3 + l) * GT + q]) * ihf[l];
          }
#pragma unroll
          for (int o = 0; o < N; ++o) {
            float s = t[off + o * STR];
#pragma unroll
            for (int j = 0; j < N; ++j) s = fmaf(tb.Dg[j * N + o], F[j], s);
            t[off + o * STR] = s;
          }
        }
    }
    __syncwarp();  // the face exchange reuses the shared region
  } else {
    // scalar: u_q kept in shared memory (private to the thread), acc in t
    float* U = tsm + cw * TpcPad<N>::UC;
#pragma unroll
    for (int q = 0; q < N3; ++q) {
      U[q] = t[q];
      const float W = tb.gw[q % N] * tb.gw[(q / N) % N] * tb.gw[q / N2] * detJ;
      t[q] *= mass * W;
    }
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const int STR = l == 0 ? 1 : (l == 1 ? N : N2);
      const float ih2 = ihf[l] * ihf[l];
#pragma unroll
      for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
          const int off = l == 0 ? (a * N + b * N2) : (l == 1 ? (a + b * N2) : (a + b * N));
          float v[N], F[N];
#pragma unroll
          for (int j = 0; j < N; ++j) v[j] = U[off + j * STR];
#pragma unroll
          for (int o = 0; o < N; ++o) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < N; ++j) s = fmaf(tb.Dg[o * N + j], v[j], s);
            const int q = off + o * STR;
            const float W = tb.gw[q % N] * tb.gw[(q / N) % N] * tb.gw[q / N2] * detJ;
            F[o] = s * W * ih2;
          }
#pragma unroll
          for (int o = 0; o < N; ++o) {
            float s = t[off + o * STR];
#pragma unroll
            for (int j = 0; j < N; ++j) s = fmaf(tb.Dg[j * N + o], F[j], s);
            t[off + o * STR] = s;
          }
        }
    }
  }
  // back to the nodes
  rsweep3<N, 0, true>(t, tb.S);
  rsweep3<N, 1, true>(t, tb.S);
  rsweep3<N, 2, true>(t, tb.S);

  // ------------------------------------------------------------- face terms
  float lam_e;
  {
    lam_e = lambda_f<TOPO>(g, e, ijk, ihf);
  }
  tpc_faces<N, NC, TOPO, 0>(g, tb, x, xe, nu_face, e, kk, cw, active, ijk, ihf, lam_e, lc, t, tsm);
  tpc_faces<N, NC, TOPO, 1>(g, tb, x, xe, nu_face, e, kk, cw, active, ijk, ihf, lam_e, lc, t, tsm);
  tpc_faces<N, NC, TOPO, 2>(g, tb, x, xe, nu_face, e, kk, cw, active, ijk, ihf, lam_e, lc, t, tsm);
  if (store) {
    float* ye = y + ((size_t)e * NC + kk) * N3;
    if constexpr (N3 % 4 == 0) {
      float4* y4 = reinterpret_cast<float4*>(ye);
#pragma unroll
      for (int i = 0; i < N3 / 4; ++i) y4[i] = make_float4(t[4 * i], t[4 * i + 1], t[4 * i + 2], t[4 * i + 3]);
    } else {
#pragma unroll
      for (int i = 0; i < N3; ++i) ye[i] = t[i];
    }
  }
}

}  // namespace sipg
