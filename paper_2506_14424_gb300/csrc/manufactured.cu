// Load vectors of the manufactured solutions used to verify the operators
// (Sec. 7.1 checks convergence with manufactured solutions; here the steady
// operators alone): b_i = integral over the cell of phi_i f, over-integrated
// with n + 3 Gauss points per direction, one CTA per cell, f evaluated at the
// points, then three transposed sweeps onto the Gauss-Lobatto basis.
//   case 0 (velocity, ncomp 3): u = s(x) c, s = sin(pi x) sin(pi y) sin(pi z),
//     c = (1, -1, 2), nu = 1 + 9 s^2 (the analytic law):
//     f_i = -2 sum_j eps_ij d_j nu - nu (c_i lap s + sum_j c_j d_i d_j s),
//     eps_ij = (c_i d_j s + c_j d_i s) / 2, d_j nu = 18 s d_j s;
//   case 1 (pressure, ncomp 1): p = cos(pi x) cos(pi y) cos(pi z), f = 3 pi^2 p.
// sin/cos come from CUDA's sincospi.
#include "../../include/sipg.h"
#include "ctx.h"
#include "kernels.cuh"
#include "sweeps.cuh"
#include "tables.h"

namespace sipg {
namespace {

using namespace sweeps;

template <int N, int NQ>
__global__ void __launch_bounds__(kSplitThreads) mms_load_kernel(LevelGeom g, LoadTab lt, int which,
                                                                 double* __restrict__ b) {
  constexpr int NQ3 = NQ * NQ * NQ, N3 = N * N * N;
  __shared__ double S[N * NQ];
  __shared__ double F[3][NQ3], T0[N * NQ * NQ], T1[N * N * NQ], OUT[N3];
  const int e = blockIdx.x;
  const int ncomp = which == 0 ? 3 : 1;
  for (int i = threadIdx.x; i < N * NQ; i += blockDim.x) S[i] = lt.S[i];
  int ijk[3];
  cell_ijk(g, e, ijk);
  const double detJ = g.h[0] * g.h[1] * g.h[2];
  const double pi = 3.141592653589793;
  for (int q = threadIdx.x; q < NQ3; q += blockDim.x) {
    const int qi[3] = {q % NQ, (q / NQ) % NQ, q / (NQ * NQ)};
    double sn[3], cs[3];
    for (int d = 0; d < 3; ++d) sincospi(g.x0[d] + (ijk[d] + lt.gp[qi[d]]) * g.h[d], &sn[d], &cs[d]);
    const double W = lt.gw[qi[0]] * lt.gw[qi[1]] * lt.gw[qi[2]] * detJ;
    if (which == 0) {
      const double c[3] = {1.0, -1.0, 2.0};
      const double s = sn[0] * sn[1] * sn[2];
      const double gr[3] = {pi * cs[0] * sn[1] * sn[2], pi * sn[0] * cs[1] * sn[2], pi * sn[0] * sn[1] * cs[2]};
      double H[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          H[i][j] = i == j ? -pi * pi * s : pi * pi * cs[i] * cs[j] * sn[3 - i - j];
      const double nu = 1.0 + 9.0 * s * s;
      const double lap = H[0][0] + H[1][1] + H[2][2];
      for (int i = 0; i < 3; ++i) {
        double f = 0.0;
        for (int j = 0; j < 3; ++j) f -= (c[i] * gr[j] + c[j] * gr[i]) * 18.0 * s * gr[j];
        double hc = 0.0;
        for (int j = 0; j < 3; ++j) hc += H[i][j] * c[j];
        f -= nu * (c[i] * lap + hc);
        F[i][q] = W * f;
      }
    } else {
      F[0][q] = W * 3.0 * pi * pi * cs[0] * cs[1] * cs[2];
    }
  }
  __syncthreads();
  for (int c = 0; c < ncomp; ++c) {
    sweep<NQ, NQ, NQ, 0, N, true>(S, N, F[c], T0);
    __syncthreads();
    sweep<N, NQ, NQ, 1, N, true>(S, N, T0, T1);
    __syncthreads();
    sweep<N, N, NQ, 2, N, true>(S, N, T1, OUT);
    __syncthreads();
    for (int i = threadIdx.x; i < N3; i += blockDim.x) b[((size_t)e * ncomp + c) * N3 + i] = OUT[i];
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_manufactured_load(int n, const LevelGeom& g, int which, double* b, cudaStream_t st) {
  if (g.ncells == 0) return cudaSuccess;
  const LoadTab lt = make_load_tab(n);
  switch (n) {
    case 2: mms_load_kernel<2, 5><<<g.ncells, kSplitThreads, 0, st>>>(g, lt, which, b); break;
    case 3: mms_load_kernel<3, 6><<<g.ncells, kSplitThreads, 0, st>>>(g, lt, which, b); break;
    case 4: mms_load_kernel<4, 7><<<g.ncells, kSplitThreads, 0, st>>>(g, lt, which, b); break;
    case 5: mms_load_kernel<5, 8><<<g.ncells, kSplitThreads, 0, st>>>(g, lt, which, b); break;
    case 6: mms_load_kernel<6, 9><<<g.ncells, kSplitThreads, 0, st>>>(g, lt, which, b); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace sipg

using namespace sipg;

extern "C" int sipg_rhs_manufactured(sipg_ctx* ctx, int case_id, double* b) {
  if (!ctx || !b || (case_id != SIPG_MMS_VELOCITY && case_id != SIPG_MMS_PRESSURE)) return SIPG_ERR_INVALID;
  if (ctx->mapped) return ctx->fail(SIPG_ERR_INVALID, "manufactured loads on affine cells only");
  const int op = case_id == SIPG_MMS_VELOCITY ? SIPG_OP_VISCOUS : SIPG_OP_POISSON;
  const Level& L = ctx->hier[op].cph ? ctx->hier[op].T[0] : ctx->hier[op].L[0];
  cudaError_t e = launch_manufactured_load(L.n, L.g, case_id, b, ctx->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  if (e != cudaSuccess) return ctx->fail(SIPG_ERR_CUDA, "manufactured load", e);
  return SIPG_OK;
}
