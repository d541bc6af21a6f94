// FP64 instantiations of the fused cell + face SIPG operator kernel.
#include "apply_dispatch.cuh"
#include "kernels.cuh"
namespace sipg {
template <>
cudaError_t launch_apply<double>(int n, int ncomp, const LevelGeom& g, const Tab& tab, const double* x, double* y,
                                 const double* nu_cell, const double* nu_face, double mass, int nbatch,
                                 cudaStream_t st) {
  return launch_apply_t<double, double, double, double>(n, ncomp, g, tab, x, y, nu_cell, nu_face, mass, nbatch, st);
}

cudaError_t launch_apply_multi_f64(int n, int ncomp, const void* descs, const int2* tiles, int ntiles,
                                   const Tab& tab, cudaStream_t st) {
  return launch_apply_multi_t<double, double, double>(n, ncomp, static_cast<const ApplyDesc<double, double>*>(descs),
                                                      tiles, ntiles, tab, st);
}
}  // namespace sipg
