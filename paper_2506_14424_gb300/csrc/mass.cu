// Cell mass matrix and its inverse (Sec. 5.1: the element-local L2 inner
// product (v, u)_{Omega_e} of Eqs. convective_step_weak, projection_step_weak
// and viscous_step_weak).
//
// On an affine box cell with the tensor-product Gauss-Lobatto basis and the
// (k+1)-point Gauss rule the block of one component factorises exactly:
//     M_e = det J (M1 (x) M1 (x) M1),   M1[i][j] = sum_q w_q l_i(g_q) l_j(g_q),
// and so does its inverse, M_e^-1 = (M1^-1 (x) M1^-1 (x) M1^-1) / det J. The
// kernel applies either as three line sweeps in shared memory: a cell's
// values are read once and written once, so the kernel is bound by HBM
// (16 bytes per DoF in FP64 storage) when the sweeps run on the FP32 pipe
// (float-float or FP32); FP64 sweeps (6 n flops per DoF) are bound by the
// FP64 pipe instead.
//
// x and y may be the same buffer: each CTA reads all values of its cells
// before it writes any of them, and CTAs own disjoint cells.
#include "ff.cuh"
#include "kernels.cuh"

#include <algorithm>

namespace sipg {
namespace {

template <int N, typename T>
struct MTab {
  T m[N * N];
};

template <int N, int NC>
struct MassCfg {
  static constexpr int V = NC * N * N * N;          // values per cell
  static constexpr int CPB = V >= 2048 ? 1 : 2048 / V;
  static constexpr int NT = 256;
};

template <typename T>
inline T host_conv(double d) { return T(d); }
template <>
inline ff host_conv<ff>(double d) {
  const float h = (float)d;
  return ff(h, (float)(d - (double)h));
}

// One 1D line of a sweep: out[i*S] = sum_m M[i][m] in[m*S], with the line's
// values in registers and M read at compile-time indices from the kernel
// parameters (constant bank operands, no shared-memory traffic for M).
template <int N, int S, typename T>
__device__ __forceinline__ void line_apply(const MTab<N, T>& mt, const T* in, T* out) {
  T v[N];
#pragma unroll
  for (int m = 0; m < N; ++m) v[m] = in[m * S];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    Acc<T> acc;
#pragma unroll
    for (int m = 0; m < N; ++m) acc.add(mt.m[i * N + m], v[m]);
    out[i * S] = acc.get();
  }
}

template <int N, int NC, typename TS, typename T>
__global__ void __launch_bounds__(MassCfg<N, NC>::NT) cell_mass_kernel(int ncells, MTab<N, T> mt, T scale,
                                                                       const TS* x, TS* y) {
  using Cfg = MassCfg<N, NC>;
  constexpr int V = Cfg::V, N2 = N * N, N3 = N2 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* B = A + Cfg::CPB * V;
  const int64_t c0 = (int64_t)blockIdx.x * Cfg::CPB;
  const int nc = (int)min((int64_t)Cfg::CPB, (int64_t)ncells - c0);
  const int tot = nc * V;
  const int64_t base = c0 * V;
  // all loads of a thread in flight before any shared-memory store
  constexpr int TOT = Cfg::CPB * V, PER = (TOT + Cfg::NT - 1) / Cfg::NT;
  TS v[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = threadIdx.x + j * Cfg::NT;
    v[j] = i < tot ? x[base + i] : TS(0);
  }
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = threadIdx.x + j * Cfg::NT;
    if (i < TOT) A[i] = stream_load<T>(v[j]);
  }
  __syncthreads();
  const int lines = tot / N;  // lines per direction in this CTA (nc * NC * N^2)
  for (int l = threadIdx.x; l < lines; l += blockDim.x)  // along x: lines are contiguous
    line_apply<N, 1, T>(mt, A + l * N, B + l * N);
  __syncthreads();
  for (int l = threadIdx.x; l < lines; l += blockDim.x) {  // along y: (component plane, ix)
    const int o = (l / N) * N2 + l % N;
    line_apply<N, N, T>(mt, B + o, A + o);
  }
  __syncthreads();
  for (int l = threadIdx.x; l < lines; l += blockDim.x) {  // along z, scaled, to global memory
    const int o = (l / N2) * N3 + l % N2;
    T w[N];
#pragma unroll
    for (int m = 0; m < N; ++m) w[m] = A[o + m * N2];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      Acc<T> acc;
#pragma unroll
      for (int m = 0; m < N; ++m) acc.add(mt.m[i * N + m], w[m]);
      y[base + o + i * N2] = stream_store<TS>(acc.get() * scale);
    }
  }
}

template <int N, int NC, typename TS, typename T>
cudaError_t launch_mass_n(int ncells, const Tab& tab, bool inverse, double scale, const TS* x, TS* y,
                          cudaStream_t st) {
  using Cfg = MassCfg<N, NC>;
  if (ncells == 0) return cudaSuccess;
  MTab<N, T> mt;
  const double* src = inverse ? tab.M1inv : tab.M1;
  for (int i = 0; i < N * N; ++i) mt.m[i] = host_conv<T>(src[i]);
  const size_t smem = 2 * sizeof(T) * Cfg::CPB * Cfg::V;
  const int grid = (ncells + Cfg::CPB - 1) / Cfg::CPB;
  cell_mass_kernel<N, NC, TS, T><<<grid, Cfg::NT, smem, st>>>(ncells, mt, host_conv<T>(scale), x, y);
  return cudaGetLastError();
}

template <typename TS, typename T>
cudaError_t launch_mass_t(int n, int ncomp, int ncells, const Tab& tab, bool inverse, double scale, const TS* x,
                          TS* y, cudaStream_t st) {
#define SIPG_MCASE(NN)                                                                                  \
  case NN:                                                                                              \
    return ncomp == 3 ? launch_mass_n<NN, 3, TS, T>(ncells, tab, inverse, scale, x, y, st)             \
                      : launch_mass_n<NN, 1, TS, T>(ncells, tab, inverse, scale, x, y, st);
  switch (n) {
    SIPG_MCASE(2)
    SIPG_MCASE(3)
    SIPG_MCASE(4)
    SIPG_MCASE(5)
    SIPG_MCASE(6)
    default: return cudaErrorInvalidValue;
  }
#undef SIPG_MCASE
}

}  // namespace

cudaError_t launch_cell_mass(int n, int ncomp, int ncells, const Tab& tab, int arith, bool inverse, double scale,
                             const void* x, void* y, cudaStream_t st) {
  switch (arith) {
    case 0:  // FP64
      return launch_mass_t<double, double>(n, ncomp, ncells, tab, inverse, scale, (const double*)x, (double*)y, st);
    case 1:  // FP32
      return launch_mass_t<float, float>(n, ncomp, ncells, tab, inverse, scale, (const float*)x, (float*)y, st);
    case 2:  // float-float, FP64 storage
      return launch_mass_t<double, ff>(n, ncomp, ncells, tab, inverse, scale, (const double*)x, (double*)y, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace sipg
