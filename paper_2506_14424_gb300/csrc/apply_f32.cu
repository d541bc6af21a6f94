// FP32 instantiations of the fused cell + face SIPG operator kernel (multigrid levels).
#include "apply_dispatch.cuh"
namespace sipg {
template cudaError_t launch_apply<float>(int, int, const LevelGeom&, const Tab&, const float*, float*,
                                         const float*, const float*, float, int,
                                          cudaStream_t);
}
