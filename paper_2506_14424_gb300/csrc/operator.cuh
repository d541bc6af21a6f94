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
// so there are no atomics and the result is deterministic. Every loop runs a
// compile-time count (CPB cells, also in the last CTA of a level, whose cells
// beyond the level's end repeat its last cell and are never stored), and the
// neighbour, boundary kind and penalty of each of the CTA's faces are looked
// up once per CTA into shared tables. Per cell:
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

#include <type_traits>

namespace sipg {

// 1D tables in the arithmetic type of a kernel (kernel parameter: compile-time
// indices become constant-bank operands, no shared-memory traffic).
template <typename T>
struct CTab {
  T S[kMaxN * kMaxN];
  T Dg[kMaxN * kMaxN];
  T dS0[kMaxN], dS1[kMaxN], gw[kMaxN];
};

// Host conversion of a binary64 value to the kernel's arithmetic type (the
// float-float split is exact: hi = RN(d), lo = RN(d - hi)).
template <typename T>
inline T host_from_double(double d) { return T(d); }
template <>
inline ff host_from_double<ff>(double d) {
  const float h = (float)d;
  return ff(h, (float)(d - (double)h));
}

// Per-level constants of one apply in the arithmetic type, converted on the
// host, so that the float-float and FP32 kernels issue no FP64 instruction
// (this GPU's FP64 pipe runs about 1/70 of the FP32 rate): 1/h per direction,
// the face area h_t1 h_t2 per normal direction, the cell volume, the mass
// coefficient and C_IP N^2 of the penalty.
template <typename T>
struct LevelConsts {
  T ih[3], area[3], detJ, mass, cipn2;
};
template <typename T>
inline LevelConsts<T> level_consts(const LevelGeom& g, int n, double mass) {
  LevelConsts<T> c;
  for (int d = 0; d < 3; ++d) c.ih[d] = host_from_double<T>(g.ih[d]);
  c.area[0] = host_from_double<T>(g.h[1] * g.h[2]);
  c.area[1] = host_from_double<T>(g.h[0] * g.h[2]);
  c.area[2] = host_from_double<T>(g.h[0] * g.h[1]);
  c.detJ = host_from_double<T>(g.h[0] * g.h[1] * g.h[2]);
  c.mass = host_from_double<T>(mass);
  c.cipn2 = host_from_double<T>(g.cip * double(n * n));
  return c;
}

// Penalty length scale of a cell in the arithmetic type: sum over its faces of
// w / h_d, w = 1/2 on interior faces and 1 on boundary faces.
template <bool TOPO, typename T>
__device__ __forceinline__ T penalty_lambda_c(const LevelGeom& g, int e, const T* ih) {
  T lam = T(0);
#pragma unroll
  for (int f = 0; f < 6; ++f) lam = lam + (cell_neighbor_t<TOPO>(g, e, f) >= 0 ? T(0.5f) : T(1)) * ih[f >> 1];
  return lam;
}

template <typename T>
__device__ __forceinline__ T nubar_of(int mode, T a, T b) {
  if (mode == 1) return T(0.5f) * (a + b);
  if (mode == 2) return T(2) * a * b / (a + b);
  return a > b ? a : b;
}

// Shared-memory swizzle of the degree-3 tensors of the binary64 kernel: inside
// each 128-byte row of 16 doubles the element index is XORed with r + 4r, r =
// row index mod 4 (the z layer of a cell tensor, the component-cell index of a
// face slot). The threads of a warp then touch every bank pair at most twice in
// the x-, y- and z-line sweeps and in the line phases of the face slots, instead
// of up to eight times (row strides of 4 and 16 elements). Every access to a
// tensor uses the same map of its index relative to the region's base (Xs, Y,
// W0..W2, the face slots F), and the bases are multiples of 16 elements.
// Measured at 32^3, k = 3: binary64 2.62 -> 2.56 ms; the float-float kernel
// (issue bound) lost more to the index arithmetic than it gained (0.787 ->
// 0.885 ms) and keeps the plain layout.
template <int N, typename T>
__device__ __forceinline__ int swz(int i) {
  if constexpr (N == 4 && std::is_same<T, double>::value) return i ^ (((i >> 4) & 3) * 5);
  else return i;
}

// out[t][.. o ..] (+)= sum_j M(o, j) in[t][.. j ..] along direction DIR of
// N^3 tensors (x fastest); M(o, j) = M[o*N + j], or M[j*N + o] if TR.
// One thread per 1D line: the N inputs are loaded once into registers, the
// N x N matrix comes from the kernel-parameter bank, N outputs are stored.
// SW: the tensors are stored with the swizzle swz (the operator kernel).
template <int N, int DIR, bool TR, bool ACC, bool SW = false, typename T>
__device__ __forceinline__ void sweep3(const T* __restrict__ in, T* __restrict__ out, const T* M, int ntens) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int STR = DIR == 0 ? 1 : (DIR == 1 ? N : N2);
  for (int line = threadIdx.x; line < ntens * N2; line += blockDim.x) {
    const int t = line / N2, r = line - t * N2;
    // r enumerates the two other coordinates, the lower one fastest
    const int off = t * N3 + (DIR == 0 ? r * N : (DIR == 1 ? (r % N) + (r / N) * N2 : r));
    T v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = in[SW ? swz<N, T>(off + j * STR) : off + j * STR];
#pragma unroll
    for (int o = 0; o < N; ++o) {
      Acc<T> acc;
#pragma unroll
      for (int j = 0; j < N; ++j) acc.add(TR ? M[j * N + o] : M[o * N + j], v[j]);
      T* dst = out + (SW ? swz<N, T>(off + o * STR) : off + o * STR);
      *dst = ACC ? *dst + acc.get() : acc.get();
    }
  }
}

// Same on N^2 face tensors (a fastest): DIR 0 along a, 1 along b.
template <int N, int DIR, bool TR, bool ACC, typename T>
__device__ __forceinline__ void sweep2(const T* __restrict__ in, T* __restrict__ out, const T* M, int ntens) {
  constexpr int N2 = N * N;
  constexpr int STR = DIR == 0 ? 1 : N;
  for (int line = threadIdx.x; line < ntens * N; line += blockDim.x) {
    const int t = line / N, r = line - t * N;
    const int off = t * N2 + (DIR == 0 ? r * N : r);
    T v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = in[off + j * STR];
#pragma unroll
    for (int o = 0; o < N; ++o) {
      Acc<T> acc;
#pragma unroll
      for (int j = 0; j < N; ++j) acc.add(TR ? M[j * N + o] : M[o * N + j], v[j]);
      T* dst = out + off + o * STR;
      *dst = ACC ? *dst + acc.get() : acc.get();
    }
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

// Cells per CTA and threads per CTA of the operator kernels (one thread per 1D
// line of a sweep). Measured at 32^3, k = 3 with the float-float arithmetic
// (1.086 / 0.964 / 0.849 / 0.838 ms for 2 / 4 / 6 / 8 cells; FP64 unchanged at
// 2.776 ms): larger CTAs amortise the barriers of the cooperative sweeps and
// keep more independent lines per warp in flight.
template <int N, int NC> struct OpCfg {
  static constexpr int CPB = NC == 3 ? (N == 2 ? 8 : (N == 3 ? 4 : (N == 4 ? 8 : (N == 5 ? 2 : 1))))
                                     : (N == 2 ? 32 : (N == 3 ? 12 : (N == 4 ? 8 : (N == 5 ? 4 : 3))));
  static constexpr int LINES = CPB * NC * N * N;
  static constexpr int NT = ((LINES + 31) / 32) * 32;
};

// Minimum resident CTAs per SM requested from the compiler, from a register
// budget per thread: the float-float and FP32 kernels are issue and latency
// bound, and more resident warps hide more of it. Measured at 32^3, k = 3:
// float-float 72 -> 56 registers 1.347 -> 1.266 ms (36 bytes of spills),
// FP32 59 -> 48 registers 0.398 -> 0.361 ms; with 8 cells per CTA a 64-register
// budget is 8 % slower than 56 (0.907 vs 0.838 ms) and 48 equal. The native FP64
// kernel is bound by the FP64 pipe and keeps MIN = 1.
#ifndef SIPG_FF_REG
#define SIPG_FF_REG 56
#endif
template <int N, int NC, typename T> struct OccCfg { static constexpr int MIN = 1; };
#ifndef SIPG_F32_REG
#define SIPG_F32_REG 48
#endif
template <int N, int NC> struct OccCfg<N, NC, float> {
  static constexpr int REG = SIPG_F32_REG;
  static constexpr int MIN = REG == 0 ? 1 : (65536 / (OpCfg<N, NC>::NT * REG) > 0 ? 65536 / (OpCfg<N, NC>::NT * REG) : 1);
};
template <int N, int NC> struct OccCfg<N, NC, ff> {
  static constexpr int REG = SIPG_FF_REG;
  static constexpr int MIN = 65536 / (OpCfg<N, NC>::NT * REG) > 0 ? 65536 / (OpCfg<N, NC>::NT * REG) : 1;
};

// Shared-memory layout (elements of T): the 1D tables, the face penalties, the
// quadrature weights times det J of the N^3 cell points, and per cell the staged
// x, the y accumulator and a work region used by the cell phase (3 tensors) and
// then by the face phase (16 face slots: 8 per side of one direction).
template <int N, int NC>
__host__ __device__ constexpr int op_work_elems() {
  return (3 * NC * N * N * N > 16 * NC * N * N) ? 3 * NC * N * N * N : 16 * NC * N * N;
}
template <int N, int NC>
__host__ __device__ constexpr int op_smem_elems() {
  return 2 * N * N + 4 * N + 6 * OpCfg<N, NC>::CPB + N * N * N +
         OpCfg<N, NC>::CPB * (2 * NC * N * N * N + op_work_elems<N, NC>());
}
// bytes: the T region above, then the per-CTA face table (int, 6 per cell):
// the neighbour across each face, or kBndDirichlet / kBndNeumann
template <int N, int NC, typename T>
__host__ __device__ constexpr size_t op_smem_bytes() {
  return ((sizeof(T) * op_smem_elems<N, NC>() + 15) / 16) * 16 + sizeof(int) * 6 * OpCfg<N, NC>::CPB;
}
constexpr int kBndDirichlet = -1, kBndNeumann = -2;

template <int N, typename T>
__device__ __forceinline__ void load_tables(const CTab<T>& ct, T* dS0, T* dS1, T* gw) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    dS0[i] = ct.dS0[i];
    dS1[i] = ct.dS1[i];
    gw[i] = ct.gw[i];
  }
}

// Numerical flux at the quadrature points of both faces of direction D of the
// CTA's cells. Per side s, slots F[s*8 + .] of FS elements hold on entry:
//   0 own trace gV, 1 own normal derivative gN, 2 neighbour trace gVp,
//   3 neighbour normal derivative gNp, 4 own d/dxi_t2 gT2, 5 own d/dxi_t1 gT1,
//   6 neighbour d/dxi_t2, 7 neighbour d/dxi_t1   (reference coordinates)
// and on exit slots 0, 1, 5, 4 hold the coefficients of the test value, of
// the normal test derivative and of the two tangential test derivatives.
// pen[s*CPB + c] = C_IP (k+1)^2 max(Lambda-, Lambda+).
template <typename T>
__device__ __forceinline__ T sel3(const T* v, int i) { return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]); }

template <int N, int NC, typename TN, typename T>
__device__ __forceinline__ void face_flux_pair(int D, const LevelGeom& g, int cell0, int FS, const T* ih,
                                               const T area, const T* gw, const T* pen, const int* nbt,
                                               const TN* __restrict__ nu_face, T* F) {
  constexpr int N2 = N * N, CPB = OpCfg<N, NC>::CPB;
  const int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;
  const T ihd = sel3(ih, D), iht1 = sel3(ih, T1), iht2 = sel3(ih, T2);
  const int last = g.ncells - 1;
  for (int i = threadIdx.x; i < 2 * CPB * N2; i += blockDim.x) {
    const int s = i / (CPB * N2);
    const int rem = i - s * CPB * N2;
    const int c = rem / N2, p = rem - c * N2;
    const int a = p % N, b = p / N;
    const int e = min(cell0 + c, last);
    const int f = 2 * D + s;
    const int nb = nbt[c * 6 + f];
    // slot q of side s, entry j
    auto at = [&](int q, int j) -> T& { return F[swz<N, T>((s * 8 + q) * FS + j)]; };
    if (nb == kBndNeumann) {  // homogeneous Neumann: no face term
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        const int j = (c * NC + k) * N2 + p;
        at(0, j) = T(0); at(1, j) = T(0);
      }
      if (NC == 3) {
        const int jd = (c * 3 + D) * N2 + p;
        at(5, jd) = T(0); at(4, jd) = T(0);
      }
      continue;
    }
    const bool inner = nb >= 0;
    const T nsign = s ? T(1) : T(-1);
    const T W = gw[a] * gw[b] * area;
    const T pe = pen[c * 6 + f];
    if constexpr (NC == 3) {
      const T num = load_as<T>(nu_face[((size_t)e * 6 + f) * N2 + p]);
      const T nup = inner ? load_as<T>(nu_face[((size_t)nb * 6 + (f ^ 1)) * N2 + p]) : num;
      const T tW = pe * nubar_of<T>(g.face_nu, num, nup) * W;  // tau W
      // Only grad u_D . e_l (l tangential) and d u_k / d x_D enter the flux:
      // P_k = tau ([u]_k + d_kD [u]_D) - sigma (A_kD + A_Dk), A = (nu- G- + nu+ G+)/2;
      // Q = -nu- sym([u] (x) n): Q_kD = -nu- sigma [u]_k (1 + d_kD)/2, Q_Dl = -nu- sigma [u]_l / 2.
      const T am = T(0.5f) * nsign * num * W;   // sigma nu-/2 W
      const T ap = T(0.5f) * nsign * nup * W;   // sigma nu+/2 W
      const T cq = -am;                          // -sigma nu-/2 W
      T um[3], nm[3], up[3], npd[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int j = (c * 3 + k) * N2 + p;
        um[k] = at(0, j);
        nm[k] = at(1, j);
        if (inner) {
          up[k] = at(2, j);
          npd[k] = at(3, j);
        } else {  // Dirichlet mirror: u+ = -u-, grad u+ = grad u-
          up[k] = -um[k];
          npd[k] = nm[k];
        }
      }
      const int jd = (c * 3 + D) * N2 + p;
      const T t1m = at(5, jd), t2m = at(4, jd);
      const T t1p = inner ? at(7, jd) : t1m;
      const T t2p = inner ? at(6, jd) : t2m;
      T jmp[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) jmp[k] = um[k] - up[k];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int j = (c * 3 + k) * N2 + p;
        if (k == D) {
          at(0, j) = T(2) * (tW * jmp[k] - (am * nm[k] + ap * npd[k]) * ihd);
          at(1, j) = T(2) * cq * jmp[k] * ihd;
        } else {
          const T tm = k == T1 ? t1m * iht1 : t2m * iht2;
          const T tp = k == T1 ? t1p * iht1 : t2p * iht2;
          at(0, j) = tW * jmp[k] - (am * (nm[k] * ihd + tm) + ap * (npd[k] * ihd + tp));
          at(1, j) = cq * jmp[k] * ihd;
        }
      }
      at(5, jd) = cq * sel3(jmp, T1) * iht1;
      at(4, jd) = cq * sel3(jmp, T2) * iht2;
    } else {
      const T tau = pe;
      const int j = c * N2 + p;
      const T pm = at(0, j);
      const T dnm = at(1, j) * ihd;
      T pp, dnp;
      if (inner) {
        pp = at(2, j);
        dnp = at(3, j) * ihd;
      } else {
        pp = -pm;
        dnp = dnm;
      }
      const T jmp = pm - pp;
      // -grad q . n jump/2 - q ({{dp/dx_d}} n_d - tau jump)
      at(0, j) = -W * (T(0.5f) * (dnm + dnp) * nsign - tau * jmp);
      at(1, j) = -W * T(0.5f) * jmp * nsign * ihd;
    }
  }
}

// 1D contraction of one line held in registers: out[o] = sum_j M(o, j) v[j]
template <int N, bool TR, typename T>
__device__ __forceinline__ T line_dot(const T* M, const T* v, int o) {
  Acc<T> acc;
#pragma unroll
  for (int j = 0; j < N; ++j) acc.add(TR ? M[j * N + o] : M[o * N + j], v[j]);
  return acc.get();
}

// Face terms of direction D (both sides) added to Y. One non-inlined copy
// serves the three directions (the direction only changes indices), which
// keeps the unrolled float-float code within the instruction cache.
// S and Dg point to shared-memory copies of the 1D matrices; nbt / pen are the
// CTA's face tables (neighbour or boundary kind, penalty factor).
template <int N, int NC, typename TX, typename TN, typename T>
__device__ __noinline__ void face_pair(int D, const LevelGeom& g, const T* S, const T* Dg, int cell0,
                                       const TX* __restrict__ x, const TN* __restrict__ nu_face, const T* Xs, T* Y,
                                       T* F, const T* pen, const int* nbt, const T* ih, const T area, const T* gw,
                                       const T* dS0, const T* dS1) {
  constexpr int N2 = N * N, N3 = N2 * N, CPB = OpCfg<N, NC>::CPB;
  constexpr int nt = CPB * NC;
  constexpr int FS = CPB * NC * N2;
  const int STD = D == 0 ? 1 : (D == 1 ? N : N2);
  // (A) traces and normal derivatives at the face Gauss-Lobatto nodes of both
  // sides (neighbour data straight from global memory)
  for (int i = threadIdx.x; i < 2 * nt * N2; i += blockDim.x) {
    const int s = i / (nt * N2);
    const int rem = i - s * nt * N2;
    const int t = rem / N2, p = rem - t * N2;
    const int c = t / NC, comp = t - c * NC;
    const int off0 = face_node<N>(D, 0, p % N, p / N);
    const T* dS = s ? dS1 : dS0;
    const T* dSn = s ? dS0 : dS1;
    const int xb = t * N3 + off0;
    Acc<T> dn;
#pragma unroll
    for (int j = 0; j < N; ++j) dn.add(dS[j], Xs[swz<N, T>(xb + j * STD)]);
    const int fb = s * 8 * FS + rem;
    F[swz<N, T>(fb)] = Xs[swz<N, T>(xb + (s ? N - 1 : 0) * STD)];
    F[swz<N, T>(fb + FS)] = dn.get();
    const int nb = nbt[c * 6 + 2 * D + s];
    if (nb >= 0) {
      const TX* xn = x + ((size_t)nb * NC + comp) * N3 + off0;
      T v[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = load_as<T>(xn[j * STD]);
      Acc<T> dnn;
#pragma unroll
      for (int j = 0; j < N; ++j) dnn.add(dSn[j], v[j]);
      F[swz<N, T>(fb + 2 * FS)] = v[s ? 0 : N - 1];
      F[swz<N, T>(fb + 3 * FS)] = dnn.get();
    } else {
      F[swz<N, T>(fb + 2 * FS)] = T(0);
      F[swz<N, T>(fb + 3 * FS)] = T(0);
    }
  }
  __syncthreads();
// (B) interpolate the four node quantities of each side along a
  for (int line = threadIdx.x; line < 2 * 4 * nt * N; line += blockDim.x) {
    const int s = line / (4 * nt * N);
    const int rem = line - s * 4 * nt * N;
    const int q = rem / (nt * N), lt = rem - q * nt * N;
    const int t = lt / N, r = lt - t * N;
    const int ib = (s * 8 + q) * FS + t * N2 + r * N;
    const int ob = ib + 4 * FS;
    T v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = F[swz<N, T>(ib + j)];
#pragma unroll
    for (int o = 0; o < N; ++o) F[swz<N, T>(ob + o)] = line_dot<N, false>(S, v, o);
  }
  __syncthreads();
  // (C) along b: values at the face Gauss points, one thread per (side, own /
  // neighbour, line): trace and normal derivative, slots 4, 5 -> 0, 1 (own) and
  // 6, 7 -> 2, 3 (neighbour); the b-derivative of the trace (slot 4 / 6) is
  // needed only for the normal component D of the velocity
  for (int line = threadIdx.x; line < 2 * 2 * nt * N; line += blockDim.x) {
    const int s = line / (2 * nt * N);
    const int rem = line - s * 2 * nt * N;
    const int q = rem / (nt * N), lt = rem - q * nt * N;
    const int t = lt / N, r = lt - t * N;
    const int fb = s * 8 * FS + t * N2 + r;
    T va[N], vb[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      va[j] = F[swz<N, T>(fb + (4 + 2 * q) * FS + j * N)];
      vb[j] = F[swz<N, T>(fb + (5 + 2 * q) * FS + j * N)];
    }
    T gv[N];
#pragma unroll
    for (int o = 0; o < N; ++o) {
      gv[o] = line_dot<N, false>(S, va, o);
      F[swz<N, T>(fb + (2 * q) * FS + o * N)] = gv[o];
      F[swz<N, T>(fb + (2 * q + 1) * FS + o * N)] = line_dot<N, false>(S, vb, o);
    }
    if (NC == 3 && t % 3 == D) {
#pragma unroll
      for (int o = 0; o < N; ++o) F[swz<N, T>(fb + (4 + 2 * q) * FS + o * N)] = line_dot<N, false>(Dg, gv, o);
    }
  }
  __syncthreads();
  // (D) along a: tangential a-derivatives of the own and neighbour traces of
  // velocity component D (no tangential derivative enters the Poisson flux)
  if (NC == 3) {
    for (int line = threadIdx.x; line < 2 * 2 * CPB * N; line += blockDim.x) {
      const int s = line / (2 * CPB * N);
      const int rem = line - s * 2 * CPB * N;
      const int q = rem / (CPB * N), lc = rem - q * CPB * N;  // q = 0 own, 1 neighbour
      const int c = lc / N, r = lc - c * N;
      const int t = c * 3 + D;
      const int ib = (s * 8 + 2 * q) * FS + t * N2 + r * N;
      const int ob = ib + 5 * FS;
      T v[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = F[swz<N, T>(ib + j)];
#pragma unroll
      for (int o = 0; o < N; ++o) F[swz<N, T>(ob + o)] = line_dot<N, false>(Dg, v, o);
    }
    __syncthreads();
  }
  // (E) numerical flux
  face_flux_pair<N, NC, TN, T>(D, g, cell0, FS, ih, area, gw, pen, nbt, nu_face, F);
  __syncthreads();
  // (F) test side, along a: slot 2 = gV + Dg_a^T gT1
  for (int line = threadIdx.x; line < 2 * nt * N; line += blockDim.x) {
    const int s = line / (nt * N);
    const int lt = line - s * nt * N;
    const int t = lt / N, r = lt - t * N;
    const int fb = s * 8 * FS + t * N2 + r * N;
    if (NC == 3 && t % 3 == D) {
      T g5[N];
#pragma unroll
      for (int j = 0; j < N; ++j) g5[j] = F[swz<N, T>(fb + 5 * FS + j)];
#pragma unroll
      for (int o = 0; o < N; ++o) F[swz<N, T>(fb + 2 * FS + o)] = F[swz<N, T>(fb + o)] + line_dot<N, true>(Dg, g5, o);
    } else {
#pragma unroll
      for (int o = 0; o < N; ++o) F[swz<N, T>(fb + 2 * FS + o)] = F[swz<N, T>(fb + o)];
    }
  }
  __syncthreads();
  // (G) along b, one thread per (side, output, line):
  // slot 6 = S_b^T (slot 2 + Dg_b^T gT2), slot 7 = S_b^T gN
  for (int line = threadIdx.x; line < 2 * 2 * nt * N; line += blockDim.x) {
    const int s = line / (2 * nt * N);
    const int rem = line - s * 2 * nt * N;
    const int q = rem / (nt * N), lt = rem - q * nt * N;
    const int t = lt / N, r = lt - t * N;
    const int fb = s * 8 * FS + t * N2 + r;
    T w[N];
    if (q == 1) {
#pragma unroll
      for (int j = 0; j < N; ++j) w[j] = F[swz<N, T>(fb + 1 * FS + j * N)];
    } else if (NC == 3 && t % 3 == D) {
      T g4[N];
#pragma unroll
      for (int j = 0; j < N; ++j) g4[j] = F[swz<N, T>(fb + 4 * FS + j * N)];
#pragma unroll
      for (int o = 0; o < N; ++o) w[o] = F[swz<N, T>(fb + 2 * FS + o * N)] + line_dot<N, true>(Dg, g4, o);
    } else {
#pragma unroll
      for (int o = 0; o < N; ++o) w[o] = F[swz<N, T>(fb + 2 * FS + o * N)];
    }
#pragma unroll
    for (int o = 0; o < N; ++o) F[swz<N, T>(fb + (6 + q) * FS + o * N)] = line_dot<N, true>(S, w, o);
  }
  __syncthreads();
  // (H) along a: node coefficients, slot 0 (value) and slot 1 (normal)
  for (int line = threadIdx.x; line < 2 * 2 * nt * N; line += blockDim.x) {
    const int s = line / (2 * nt * N);
    const int rem = line - s * 2 * nt * N;
    const int q = rem / (nt * N), lt = rem - q * nt * N;
    const int t = lt / N, r = lt - t * N;
    const int ob = (s * 8 + q) * FS + t * N2 + r * N;
    const int ib = ob + 6 * FS;
    T v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = F[swz<N, T>(ib + j)];
#pragma unroll
    for (int o = 0; o < N; ++o) F[swz<N, T>(ob + o)] = line_dot<N, true>(S, v, o);
  }
  __syncthreads();
  // (I) scatter onto the cell nodes: value on the face layer, normal
  // derivative spread along D, both sides
  for (int i = threadIdx.x; i < nt * N3; i += blockDim.x) {
    const int t = i / N3, r = i - t * N3;
    const int ix = r % N, iy = (r / N) % N, iz = r / N2;
    const int id = D == 0 ? ix : (D == 1 ? iy : iz);
    const int fp = t * N2 + (D == 0 ? iy : ix) + N * (D == 2 ? iy : iz);
    T v = dS0[id] * F[swz<N, T>(1 * FS + fp)] + dS1[id] * F[swz<N, T>(9 * FS + fp)];
    if (id == 0) v += F[swz<N, T>(fp)];
    if (id == N - 1) v += F[swz<N, T>(8 * FS + fp)];
    Y[swz<N, T>(i)] += v;
  }
  __syncthreads();
}

// y = (m M + A) x on the cells [cell0, cell0 + CPB) of a level, executed by
// one CTA with shared memory sm (op_smem_bytes<N, NC, T>() bytes).
// NC = 3: viscous operator (nu_cell [C][N^3], nu_face [C][6][N^2]);
// NC = 1: Poisson operator (nu pointers unused).
// TX is the storage type of x, TS that of y, TN that of nu, T the arithmetic
// type (double, float, or ff = float-float: x and nu pre-split into (hi, lo)
// pairs, y stored as binary64).
template <int N, int NC, typename TX, typename TS, typename TN, typename T, bool TOPO>
__device__ __forceinline__ void apply_cells(const LevelGeom& g, const CTab<T>& ct, const LevelConsts<T>& lc,
                                            const TX* __restrict__ x, TS* __restrict__ y,
                                            const TN* __restrict__ nu_cell, const TN* __restrict__ nu_face,
                                            int cell0, unsigned char* smraw) {
  constexpr int N2 = N * N, N3 = N2 * N, CPB = OpCfg<N, NC>::CPB;
  constexpr int nt = CPB * NC;
  T* sm = reinterpret_cast<T*>(smraw);
  int* nbt = reinterpret_cast<int*>(smraw + ((sizeof(T) * op_smem_elems<N, NC>() + 15) / 16) * 16);
  T* Ssh = sm;                     // N2, copies of the 1D matrices for the face routine
  T* Dsh = Ssh + N2;               // N2
  T* dS0 = Dsh + N2;
  T* dS1 = dS0 + N;
  T* gw = dS1 + N;
  T* pen = gw + 2 * N;             // 6 * CPB: C_IP N^2 max(Lambda-, Lambda+) per face
  T* Wq = pen + 6 * CPB;           // N3: w_x w_y w_z det J of the cell points
  T* Xs = Wq + N3;                 // CPB * NC * N3
  static_assert((2 * N2 + 4 * N + 6 * CPB + N3) % 16 == 0 || N != 4, "swizzled tensors start on 128-byte rows");
  T* Y = Xs + CPB * NC * N3;       // CPB * NC * N3
  T* Wk = Y + CPB * NC * N3;       // CPB * op_work_elems
  T* W0 = Wk;
  T* W1 = Wk + CPB * NC * N3;
  T* W2 = Wk + 2 * CPB * NC * N3;
  const T* S = ct.S;
  const T* Dg = ct.Dg;

  load_tables<N>(ct, dS0, dS1, gw);
  for (int i = threadIdx.x; i < N2; i += blockDim.x) {
    Ssh[i] = ct.S[i];
    Dsh[i] = ct.Dg[i];
  }
  const int last = g.ncells - 1;
  const T ih[3] = {lc.ih[0], lc.ih[1], lc.ih[2]};
  // face tables: neighbour (or boundary kind) and penalty of each face
  for (int i = threadIdx.x; i < 6 * CPB; i += blockDim.x) {
    const int c = i / 6, f = i - 6 * c;
    const int e = min(cell0 + c, last);
    const int nb = cell_neighbor_t<TOPO>(g, e, f);
    nbt[i] = nb >= 0 ? nb : (face_bc_t<TOPO>(g, e, f) == 1 ? kBndNeumann : kBndDirichlet);
    const T lm = penalty_lambda_c<TOPO, T>(g, e, ih);
    const T lp = nb >= 0 ? penalty_lambda_c<TOPO, T>(g, nb, ih) : lm;
    pen[i] = lc.cipn2 * (lm > lp ? lm : lp);
  }
  const T mass = lc.mass;
  for (int q = threadIdx.x; q < N3; q += blockDim.x) Wq[q] = ct.gw[q % N] * ct.gw[(q / N) % N] * ct.gw[q / N2] * lc.detJ;
  const int ncell = min(CPB, g.ncells - cell0);  // cells stored by this CTA
  for (int i = threadIdx.x; i < nt * N3; i += blockDim.x) {
    const int c = i / (NC * N3);
    const int e = min(cell0 + c, last);
    Xs[swz<N, T>(i)] = load_as<T>(x[(size_t)e * NC * N3 + (i - c * NC * N3)]);
  }
  __syncthreads();

  // ---- cell term: nodes -> Gauss points along x, y; the z pass also forms
  // the collocation z-derivative
  sweep3<N, 0, false, false, true>(Xs, W1, S, nt);
  __syncthreads();
  sweep3<N, 1, false, false, true>(W1, W2, S, nt);
  __syncthreads();
  for (int line = threadIdx.x; line < nt * N2; line += blockDim.x) {
    const int t = line / N2, r = line - t * N2;
    const int off = t * N3 + r;
    T v[N], u[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = W2[swz<N, T>(off + j * N2)];
#pragma unroll
    for (int o = 0; o < N; ++o) {
      u[o] = line_dot<N, false>(S, v, o);
      W0[swz<N, T>(off + o * N2)] = u[o];
    }
#pragma unroll
    for (int o = 0; o < N; ++o) Y[swz<N, T>(off + o * N2)] = line_dot<N, false>(Dg, u, o);  // d/dz (Y free until the end)
  }
  __syncthreads();
  sweep3<N, 0, false, false, true>(W0, W1, Dg, nt);
  sweep3<N, 1, false, false, true>(W0, W2, Dg, nt);
  __syncthreads();
  if constexpr (NC == 3) {
    // 2 nu eps(u) W at the points, one thread per (cell, item, point): items
    // 0..5 the symmetric pairs (k, l), k <= l, of the gradient (each reads and
    // writes only its own two entries), items 6..8 the mass term of component
    // k - an even split of the point work over the CTA's threads
    for (int i = threadIdx.x; i < CPB * 9 * N3; i += blockDim.x) {
      const int c = i / (9 * N3), rem = i - c * 9 * N3;
      const int it = rem / N3, q = rem - it * N3;
      const T W = Wq[q];
      if (it >= 6) {
        W0[swz<N, T>((c * 3 + it - 6) * N3 + q)] *= mass * W;
        continue;
      }
      const int k = it < 3 ? it : (it == 5 ? 1 : 0);
      const int l = it < 3 ? it : (it == 3 ? 1 : 2);
      const T nuW = load_as<T>(nu_cell[(size_t)min(cell0 + c, last) * N3 + q]) * W;
      T* Bk = k == 0 ? W1 : (k == 1 ? W2 : Y);
      T* Bl = l == 0 ? W1 : (l == 1 ? W2 : Y);
      const T ihk = sel3(ih, k), ihl = sel3(ih, l);
      if (k == l) {
        // 2 nu W d_k u_k / h_k^2
        T& g = Bk[swz<N, T>((c * 3 + k) * N3 + q)];
        g = T(2) * nuW * g * ihk * ihk;
      } else {
        // e_kl = nu W (d_l u_k / h_l + d_k u_l / h_k), the same for both entries
        T& gkl = Bl[swz<N, T>((c * 3 + k) * N3 + q)];
        T& glk = Bk[swz<N, T>((c * 3 + l) * N3 + q)];
        const T e = nuW * (gkl * ihl + glk * ihk);
        gkl = e * ihl;
        glk = e * ihk;
      }
    }
  } else {
    for (int i = threadIdx.x; i < CPB * N3; i += blockDim.x) {
      const int c = i / N3, q = i - c * N3;
      const T W = Wq[q];
      T* Bl[3] = {W1, W2, Y};
      const int j = swz<N, T>(c * N3 + q);
#pragma unroll
      for (int l = 0; l < 3; ++l) Bl[l][j] = Bl[l][j] * ih[l] * W * ih[l];
      W0[j] *= mass * W;
    }
  }
  __syncthreads();
  // transposed: W0 += Dx^T W1 + Dy^T W2 + Dz^T Y, then S^T in z (fused), y, x
  sweep3<N, 0, true, true, true>(W1, W0, Dg, nt);
  __syncthreads();
  sweep3<N, 1, true, true, true>(W2, W0, Dg, nt);
  __syncthreads();
  for (int line = threadIdx.x; line < nt * N2; line += blockDim.x) {
    const int t = line / N2, r = line - t * N2;
    const int off = t * N3 + r;
    T v[N], z[N];
#pragma unroll
    for (int j = 0; j < N; ++j) z[j] = Y[swz<N, T>(off + j * N2)];
#pragma unroll
    for (int o = 0; o < N; ++o) v[o] = W0[swz<N, T>(off + o * N2)] + line_dot<N, true>(Dg, z, o);
#pragma unroll
    for (int o = 0; o < N; ++o) W1[swz<N, T>(off + o * N2)] = line_dot<N, true>(S, v, o);
  }
  __syncthreads();
  sweep3<N, 1, true, false, true>(W1, W2, S, nt);
  __syncthreads();
  sweep3<N, 0, true, false, true>(W2, Y, S, nt);  // Y = cell contribution to y
  __syncthreads();

  // ---- face terms, both faces of one direction at a time (work region reused)
  for (int d = 0; d < 3; ++d)
    face_pair<N, NC, TX, TN, T>(d, g, Ssh, Dsh, cell0, x, nu_face, Xs, Y, Wk, pen, nbt, ih, lc.area[d], gw, dS0,
                                dS1);
  const size_t base0 = (size_t)cell0 * NC * N3;
  for (int i = threadIdx.x; i < ncell * NC * N3; i += blockDim.x) y[base0 + i] = stream_store<TS>(Y[swz<N, T>(i)]);
}

// One CTA per CPB consecutive cells of one level; blockIdx.y selects one of
// several vectors applied in the same launch (columns of a batch). TOPO: the
// level has topology tables (removed cells or periodic directions).
template <int N, int NC, typename TX, typename TS, typename TN, typename T, bool TOPO>
__global__ void __launch_bounds__(OpCfg<N, NC>::NT, (OccCfg<N, NC, T>::MIN))
apply_kernel(LevelGeom g, CTab<T> ct, LevelConsts<T> lc, const TX* __restrict__ x, TS* __restrict__ y,
             const TN* __restrict__ nu_cell, const TN* __restrict__ nu_face, int64_t batch_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  x += (int64_t)blockIdx.y * batch_stride;
  y += (int64_t)blockIdx.y * batch_stride;
  apply_cells<N, NC, TX, TS, TN, T, TOPO>(g, ct, lc, x, y, nu_cell, nu_face, blockIdx.x * OpCfg<N, NC>::CPB,
                                          smem_raw);
}

// Operator applies of several problems of the same degree in one persistent
// launch: tile i = (problem, first cell) of tiles[]; CTAs stride over the
// tile list (static round robin, deterministic: every tile is computed by
// exactly the same code as in apply_kernel, so results are bitwise equal).
// The served problems are plain boxes (no topology tables) with binary64 x.
template <typename TS, typename TN>
struct ApplyDesc {
  LevelGeom g;
  LevelConsts<TN> lc;  // in the arithmetic type, which is that of nu
  const TS* x;
  TS* y;
  const TN* nu_cell;
  const TN* nu_face;
};

template <int N, int NC, typename TS, typename TN, typename T>
__global__ void __launch_bounds__(OpCfg<N, NC>::NT, (OccCfg<N, NC, T>::MIN))
apply_multi_kernel(const ApplyDesc<TS, TN>* __restrict__ descs, const int2* __restrict__ tiles, int ntiles,
                   CTab<T> ct) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int2 tl = tiles[tile];
    static_assert(std::is_same<TN, T>::value, "served applies compute in the type of nu");
    const ApplyDesc<TS, TN> d = descs[tl.x];
    apply_cells<N, NC, TS, TS, TN, T, false>(d.g, ct, d.lc, d.x, d.y, d.nu_cell, d.nu_face, tl.y, smem_raw);
    __syncthreads();  // the next tile reuses the shared memory
  }
}

}  // namespace sipg
