// FP64-accurate instantiations of the operator kernel with float-float
// arithmetic (FP64 storage of x, y and nu; pairs of FP32 in the computation).
#include "apply_dispatch.cuh"

#include <algorithm>
namespace sipg {
cudaError_t launch_apply_ff(int n, int ncomp, const LevelGeom& g, const Tab& tab, const double* x, double* y,
                            const float2* nu_cell, const float2* nu_face, double mass, int nbatch, cudaStream_t st) {
  return launch_apply_t<double, ff, ff>(n, ncomp, g, tab, x, y, reinterpret_cast<const ff*>(nu_cell),
                                        reinterpret_cast<const ff*>(nu_face), mass, nbatch, st);
}

// nu split into (hi, lo) pairs for the float-float kernels
__global__ void split_ff_kernel(int64_t n, const double* __restrict__ in, float2* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const ff v(in[i]);
    out[i] = make_float2(v.hi, v.lo);
  }
}
cudaError_t launch_split_ff(int64_t n, const double* in, float2* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  split_ff_kernel<<<blocks, 256, 0, st>>>(n, in, out);
  return cudaGetLastError();
}
}  // namespace sipg
