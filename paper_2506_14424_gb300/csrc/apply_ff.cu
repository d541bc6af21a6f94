// FP64-accurate instantiations of the operator kernel with float-float
// arithmetic (FP64 storage of x, y and nu; pairs of FP32 in the computation).
#include "apply_dispatch.cuh"

#include <algorithm>
namespace sipg {
cudaError_t launch_apply_ff(int n, int ncomp, const LevelGeom& g, const Tab& tab, const float2* x, double* y,
                            const float2* nu_cell, const float2* nu_face, double mass, int nbatch, cudaStream_t st) {
  return launch_apply_t<ff, double, ff, ff>(n, ncomp, g, tab, reinterpret_cast<const ff*>(x), y,
                                            reinterpret_cast<const ff*>(nu_cell),
                                            reinterpret_cast<const ff*>(nu_face), mass, nbatch, st);
}

cudaError_t launch_apply_multi_ff(int n, int ncomp, const void* descs, const int2* tiles, int ntiles,
                                  const Tab& tab, cudaStream_t st) {
  return launch_apply_multi_t<double, ff, ff>(n, ncomp, static_cast<const ApplyDesc<double, ff>*>(descs), tiles,
                                              ntiles, tab, st);
}

int op_cells_per_cta(int n, int ncomp) {
  switch (n) {
    case 2: return ncomp == 3 ? OpCfg<2, 3>::CPB : OpCfg<2, 1>::CPB;
    case 3: return ncomp == 3 ? OpCfg<3, 3>::CPB : OpCfg<3, 1>::CPB;
    case 4: return ncomp == 3 ? OpCfg<4, 3>::CPB : OpCfg<4, 1>::CPB;
    case 5: return ncomp == 3 ? OpCfg<5, 3>::CPB : OpCfg<5, 1>::CPB;
    case 6: return ncomp == 3 ? OpCfg<6, 3>::CPB : OpCfg<6, 1>::CPB;
    default: return 1;
  }
}

// nu split into (hi, lo) pairs for the float-float kernels
__global__ void split_ff_kernel(int64_t n, const double* __restrict__ in, float2* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const ff v(in[i]);
    out[i] = make_float2(v.hi, v.lo);
  }
}
// integer float-float conversions of the streaming kernels, exposed for their test
__global__ void ff_convert_kernel(int64_t n, const double* __restrict__ in, float2* __restrict__ hilo,
                                  double* __restrict__ back) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const ff v = stream_load<ff, double>(in[i]);
    hilo[i] = make_float2(v.hi, v.lo);
    back[i] = stream_store<double, ff>(v);
  }
}
cudaError_t launch_ff_convert(int64_t n, const double* in, float2* hilo, double* back, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  ff_convert_kernel<<<blocks, 256, 0, st>>>(n, in, hilo, back);
  return cudaGetLastError();
}

// x of the float-float operator, split once per apply with the integer
// conversion (no FP64-pipe instructions; the same bits as the hardware split)
__global__ void split_ff_int_kernel(int64_t n, const double* __restrict__ in, float2* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const ff v = split_double(in[i]);
    out[i] = make_float2(v.hi, v.lo);
  }
}
cudaError_t launch_split_ff_int(int64_t n, const double* in, float2* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  split_ff_int_kernel<<<blocks, 256, 0, st>>>(n, in, out);
  return cudaGetLastError();
}

cudaError_t launch_split_ff(int64_t n, const double* in, float2* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  split_ff_kernel<<<blocks, 256, 0, st>>>(n, in, out);
  return cudaGetLastError();
}
}  // namespace sipg
