// FP64-accurate instantiations of the operator kernel with float-float
// arithmetic (FP64 storage of x, y and nu; pairs of FP32 in the computation).
#include "apply_dispatch.cuh"
namespace sipg {
cudaError_t launch_apply_ff(int n, int ncomp, const LevelGeom& g, const Tab& tab, const double* x, double* y,
                            const double* nu_cell, const double* nu_face, double mass, int nbatch, cudaStream_t st) {
  return launch_apply_t<double, ff>(n, ncomp, g, tab, x, y, nu_cell, nu_face, mass, nbatch, st);
}
}  // namespace sipg
