// Allocation-free variant of sipg_apply_host.
//
// sipg_apply_host stages the caller's host vectors in device buffers that the
// context allocates with cudaMalloc on first use (and again when a larger
// level is applied). Some callers cannot allow that: code that runs while a
// CUDA memory pool or a framework's caching allocator owns the device memory
// budget, hosts that forbid late device allocations after start-up, or
// plain-C programs that only hold host memory and must not trigger device
// allocations from inside a library call. sipg_apply_host_static serves them:
// it stages x and y in one file-scope device array of fixed size instead.
//
// Limits and sharing rules (also stated in include/sipg.h):
//  * at most kStaticMaxDofs values per vector (the level-0 DoFs of the
//    operator); larger requests are rejected with SIPG_ERR_INVALID;
//  * the array is reserved on every GPU that loads the library, for the life
//    of the process (8 MiB);
//  * every call on a device uses the same array: calls whose work overlaps on
//    the GPU (other streams, other threads) race and must be serialised by the
//    caller. The staging halves are fully overwritten by each call (x by the
//    host-to-device copy, y by the operator), so nothing needs clearing;
//  * the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress; make that first call before any stream capture;
//  * the device that was current at sipg_create must be current at the call
//    (the array and the context's stream both belong to it); otherwise the
//    call returns SIPG_ERR_INVALID without touching any memory.
#include "../../include/sipg.h"
#include "ctx.h"

#include <mutex>

namespace {

constexpr int64_t kStaticMaxDofs = int64_t(1) << 19;  // 524,288 doubles per vector
constexpr int kMaxDevices = 64;

// x staging in the first half, y in the second.
__device__ __align__(256) double g_apply_staging[2 * kStaticMaxDofs];

std::mutex g_mu;
double* g_staging_addr[kMaxDevices] = {nullptr};

// Device address of the staging array on device `dev`, which must be the
// current device (looked up once per device; in host code the symbol itself is
// only a host-side stand-in).
cudaError_t staging_address(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_staging_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_apply_staging);
    if (e != cudaSuccess) return e;
    g_staging_addr[dev] = static_cast<double*>(p);
  }
  *out = g_staging_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int sipg_apply_host_static(sipg_ctx* ctx, int op, const double* x_host, double* y_host,
                                      double mass_coeff) {
  if (!ctx || !x_host || !y_host) return SIPG_ERR_INVALID;
  if (op != SIPG_OP_VISCOUS && op != SIPG_OP_POISSON) return ctx->fail(SIPG_ERR_INVALID, "unknown operator");
  if (op == SIPG_OP_VISCOUS && !ctx->have_nu) return ctx->fail(SIPG_ERR_STATE, "set the viscosity first");
  const int64_t n = ctx->hier[op].L[0].ndofs;
  if (n > kStaticMaxDofs)
    return ctx->fail(SIPG_ERR_INVALID,
                     "sipg_apply_host_static: vector larger than the static staging area (524288 values)");
  // The staging array is per device and the context's stream belongs to its
  // device: a call made while another device is current is refused.
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return ctx->fail(SIPG_ERR_CUDA, "cudaGetDevice", e);
  if (cur != ctx->device)
    return ctx->fail(SIPG_ERR_INVALID, "sipg_apply_host_static: the current device is not the context's device");
  double* dx = nullptr;
  e = staging_address(cur, &dx);
  if (e != cudaSuccess) return ctx->fail(SIPG_ERR_CUDA, "cudaGetSymbolAddress(staging)", e);
  double* dy = dx + kStaticMaxDofs;
  e = cudaMemcpyAsync(dx, x_host, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st);
  if (e != cudaSuccess) return ctx->fail(SIPG_ERR_CUDA, "copy x to the staging area", e);
  int rc = ctx->krylov_apply(op, dx, dy, mass_coeff);
  if (rc) return rc;
  e = cudaMemcpyAsync(y_host, dy, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  if (e != cudaSuccess) return ctx->fail(SIPG_ERR_CUDA, "copy y from the staging area", e);
  return SIPG_OK;
}
