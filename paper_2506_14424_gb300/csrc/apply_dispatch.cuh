// Runtime dispatch of (degree, components) to the operator kernel template.
#pragma once
#include "kernels.cuh"
#include "operator.cuh"

#include <algorithm>

namespace sipg {

template <typename T>
CTab<T> make_ctab(const Tab& t) {
  CTab<T> c{};
  for (int i = 0; i < kMaxN * kMaxN; ++i) {
    c.S[i] = host_from_double<T>(t.S[i]);
    c.Dg[i] = host_from_double<T>(t.Dg[i]);
  }
  for (int i = 0; i < kMaxN; ++i) {
    c.dS0[i] = host_from_double<T>(t.dS0[i]);
    c.dS1[i] = host_from_double<T>(t.dS1[i]);
    c.gw[i] = host_from_double<T>(t.gw[i]);
  }
  return c;
}

template <int N, int NC, typename TX, typename TS, typename TN, typename TC, bool TOPO>
cudaError_t launch_apply_g(const LevelGeom& g, const Tab& tab, const TX* x, TS* y, const TN* nu_cell,
                           const TN* nu_face, double mass, int nbatch, cudaStream_t st) {
  using Cfg = OpCfg<N, NC>;
  const size_t smem = op_smem_bytes<N, NC, TC>();
  static bool attr_set = false;  // per instantiation, per process (single device)
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(apply_kernel<N, NC, TX, TS, TN, TC, TOPO>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int grid = (g.ncells + Cfg::CPB - 1) / Cfg::CPB;
  if (grid == 0 || nbatch == 0) return cudaSuccess;
  const int64_t stride = (int64_t)g.ncells * NC * N * N * N;
  apply_kernel<N, NC, TX, TS, TN, TC, TOPO><<<dim3(grid, nbatch), Cfg::NT, smem, st>>>(
      g, make_ctab<TC>(tab), level_consts<TC>(g, N, mass), x, y, nu_cell, nu_face, stride);
  return cudaGetLastError();
}

// the plain box (no topology tables) keeps the arithmetic neighbour path
template <int N, int NC, typename TX, typename TS, typename TN, typename TC>
cudaError_t launch_apply_n(const LevelGeom& g, const Tab& tab, const TX* x, TS* y, const TN* nu_cell,
                           const TN* nu_face, double mass, int nbatch, cudaStream_t st) {
  return g.nbr ? launch_apply_g<N, NC, TX, TS, TN, TC, true>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st)
               : launch_apply_g<N, NC, TX, TS, TN, TC, false>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st);
}

// TX: storage of x (TS, or ff pairs for the float-float kernel), TS: of y
template <typename TX, typename TS, typename TN, typename TC>
cudaError_t launch_apply_t(int n, int ncomp, const LevelGeom& g, const Tab& tab, const TX* x, TS* y,
                           const TN* nu_cell, const TN* nu_face, double mass, int nbatch, cudaStream_t st) {
#define SIPG_CASE(NN)                                                                                         \
  case NN:                                                                                                    \
    return ncomp == 3 ? launch_apply_n<NN, 3, TX, TS, TN, TC>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st) \
                      : launch_apply_n<NN, 1, TX, TS, TN, TC>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st);
  switch (n) {
    SIPG_CASE(2)
    SIPG_CASE(3)
    SIPG_CASE(4)
    SIPG_CASE(5)
    SIPG_CASE(6)
    default:
      return cudaErrorInvalidValue;
  }
#undef SIPG_CASE
}

template <int N, int NC, typename TS, typename TN, typename TC>
cudaError_t launch_apply_multi_n(const ApplyDesc<TS, TN>* descs, const int2* tiles, int ntiles, const Tab& tab,
                                 cudaStream_t st) {
  using Cfg = OpCfg<N, NC>;
  const size_t smem = op_smem_bytes<N, NC, TC>();
  static int resident = 0;  // CTAs per SM (per instantiation, single device)
  if (resident == 0) {
    cudaError_t e = cudaFuncSetAttribute(apply_multi_kernel<N, NC, TS, TN, TC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, apply_multi_kernel<N, NC, TS, TN, TC>, Cfg::NT,
                                                        smem);
    if (e != cudaSuccess) return e;
    if (resident < 1) resident = 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(ntiles, std::max(1, sms) * resident);
  if (grid <= 0) return cudaSuccess;
  apply_multi_kernel<N, NC, TS, TN, TC><<<grid, Cfg::NT, smem, st>>>(descs, tiles, ntiles, make_ctab<TC>(tab));
  return cudaGetLastError();
}

template <typename TS, typename TN, typename TC>
cudaError_t launch_apply_multi_t(int n, int ncomp, const ApplyDesc<TS, TN>* descs, const int2* tiles, int ntiles,
                                 const Tab& tab, cudaStream_t st) {
#define SIPG_CASE(NN)                                                                                     \
  case NN:                                                                                                \
    return ncomp == 3 ? launch_apply_multi_n<NN, 3, TS, TN, TC>(descs, tiles, ntiles, tab, st)            \
                      : launch_apply_multi_n<NN, 1, TS, TN, TC>(descs, tiles, ntiles, tab, st);
  switch (n) {
    SIPG_CASE(2)
    SIPG_CASE(3)
    SIPG_CASE(4)
    SIPG_CASE(5)
    SIPG_CASE(6)
    default:
      return cudaErrorInvalidValue;
  }
#undef SIPG_CASE
}

}  // namespace sipg
