// Runtime dispatch of (degree, components) to the operator kernel template.
#pragma once
#include "kernels.cuh"
#include "operator.cuh"

namespace sipg {

template <int N, int NC, typename TS, typename TC>
cudaError_t launch_apply_n(const LevelGeom& g, const Tab& tab, const TS* x, TS* y, const TS* nu_cell,
                           const TS* nu_face, double mass, int nbatch, cudaStream_t st) {
  constexpr int CPB = OpCfg<N>::CPB;
  static_assert(sizeof(TC) == sizeof(TS) || sizeof(TC) == 8, "compute type width");
  const size_t smem = sizeof(TC) * op_smem_elems<N, NC>();
  static bool attr_set = false;  // per instantiation, per process (single device)
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(apply_kernel<N, NC, TS, TC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int grid = (g.ncells + CPB - 1) / CPB;
  if (grid == 0 || nbatch == 0) return cudaSuccess;
  const int64_t stride = (int64_t)g.ncells * NC * N * N * N;
  apply_kernel<N, NC, TS, TC><<<dim3(grid, nbatch), OpCfg<N>::NT, smem, st>>>(g, tab, x, y, nu_cell, nu_face,
                                                                              mass, stride);
  return cudaGetLastError();
}

template <typename TS, typename TC>
cudaError_t launch_apply_t(int n, int ncomp, const LevelGeom& g, const Tab& tab, const TS* x, TS* y,
                           const TS* nu_cell, const TS* nu_face, double mass, int nbatch, cudaStream_t st) {
#define SIPG_CASE(NN)                                                                                   \
  case NN:                                                                                              \
    return ncomp == 3 ? launch_apply_n<NN, 3, TS, TC>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st) \
                      : launch_apply_n<NN, 1, TS, TC>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st);
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
