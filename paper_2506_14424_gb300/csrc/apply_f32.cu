// FP32 instantiations of the fused cell + face SIPG operator kernel (multigrid levels).
#include "apply_dispatch.cuh"
namespace sipg {
template <>
cudaError_t launch_apply<float>(int n, int ncomp, const LevelGeom& g, const Tab& tab, const float* x, float* y,
                                const float* nu_cell, const float* nu_face, float mass, int nbatch,
                                cudaStream_t st) {
  return launch_apply_t<float, float, float>(n, ncomp, g, tab, x, y, nu_cell, nu_face, (double)mass, nbatch, st);
}
}  // namespace sipg
