// FP64 instantiations of the fused cell + face SIPG operator kernel.
#include "apply_dispatch.cuh"
namespace sipg {
template cudaError_t launch_apply<double>(int, int, const LevelGeom&, const Tab&, const double*, double*,
                                          const double*, const double*, double, int,
                                          cudaStream_t);
}
