// FP32 instantiations of the fused cell + face SIPG operator kernel (multigrid levels).
#include "apply_dispatch.cuh"

#include <cstdlib>
#include <cstring>
namespace sipg {
template <>
cudaError_t launch_apply<float>(int n, int ncomp, const LevelGeom& g, const Tab& tab, const float* x, float* y,
                                const float* nu_cell, const float* nu_face, float mass, int nbatch,
                                cudaStream_t st) {
  // degrees 1..3: the register-tiled kernel (operator_tpc.cuh); higher degrees, or
  // SIPG_F32_OPERATOR=shared in the environment: the shared-memory kernel
  static const bool shared_only = [] {
    const char* v = std::getenv("SIPG_F32_OPERATOR");
    return v && std::strcmp(v, "shared") == 0;
  }();
  if (!shared_only && tpc_supported(n))
    return launch_apply_tpc(n, ncomp, g, tab, x, y, nu_cell, nu_face, mass, nbatch, st);
  return launch_apply_t<float, float, float, float>(n, ncomp, g, tab, x, y, nu_cell, nu_face, (double)mass, nbatch, st);
}
}  // namespace sipg
