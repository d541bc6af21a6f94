// FMA throughput of the device's FP64 and FP32 pipes (the ALU denominators of
// the roofline fractions the benchmark reports).
//
// Every thread runs kChains independent multiply-add chains for `iters`
// iterations, so the pipe never waits on a dependency; the grid fills every
// SM several times over. The chains are x <- x * a + b with |a| < 1, which stay
// finite, and one thread per block writes a value that depends on all of them,
// so the compiler keeps every instruction. Timed with CUDA events on a
// private stream after one warm-up launch.
#include "../../include/sipg.h"

#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_chain_kernel(int iters, T a, T b, T* out) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = T(threadIdx.x + c) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = v[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == T(-12345.0)) out[blockIdx.x] = s;  // never true; keeps the chains live
}

template <typename T>
int measure(double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SIPG_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SIPG_ERR_CUDA;
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 1 << 10 : 1 << 15;
  T* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SIPG_ERR_CUDA;
  float ms = 0.f;
  if (cudaMalloc(&out, sizeof(T) * blocks) != cudaSuccess) return SIPG_ERR_NOMEM;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
      cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    fma_chain_kernel<T><<<blocks, threads, 0, st>>>(iters, T(0.999), T(1e-4), out);  // warm-up
    cudaEventRecord(e0, st);
    fma_chain_kernel<T><<<blocks, threads, 0, st>>>(iters, T(0.999), T(1e-4), out);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0) {
      const double fmas = (double)blocks * threads * iters * kChains;
      *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
      rc = SIPG_OK;
    }
  }
  if (cudaGetLastError() != cudaSuccess) rc = SIPG_ERR_CUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  return rc;
}

}  // namespace

extern "C" int sipg_alu_peak(int prec, double* tflops) {
  if (!tflops) return SIPG_ERR_INVALID;
  if (prec == SIPG_F64) return measure<double>(tflops);
  if (prec == SIPG_F32) return measure<float>(tflops);
  return SIPG_ERR_INVALID;
}
