// Divergence and continuity penalty step (Sec. 3.2, Eq. penalty_step, the last
// sub-step of Alg. 1): the velocity of the viscous step u is post-processed by
//     (v, u~) + (div v, tau_div,e div u~) + (v.n, tau_F (u~^- - u~^+).n)_dOmega_e
//       = (v, u),
// tau_F the mean of the two cells' tau_cont on interior faces and the cell's own
// on a Dirichlet wall, where the exterior state is the wall velocity g (its part
// moves to the right-hand side); Neumann walls carry no term. Penalty
// parameters per cell (the paper takes them from Fehn et al. 2018, whose formulas
// it does not print; this library's reading):
//     tau_div,e = zeta_div ubar_e h_e / (k+1) dt,  tau_cont,e = zeta_cont ubar_e dt,
// ubar_e the cell mean of |u| and h_e = |Omega_e|^(1/3).
//
// Kernels (FP64, one CTA per cell, each CTA writes only its own rows):
//   pen_tau_kernel    ubar_e by Gauss quadrature -> tau_div,e, tau_cont,e
//   pen_apply_kernel  y = K x (cell mass + div-div + normal-jump terms)
//   pen_wall_kernel   y += (v.n, tau_cont,e g.n) over Dirichlet walls
// On affine grid cells the face normal is +-e_d, so the jump term acts on component d
// only, on the face layer of Gauss-Lobatto coefficients (the trace of the
// nodal basis). The system is symmetric positive definite and close to the
// mass matrix (the penalties scale with the Courant number), so it is solved
// by CG preconditioned with the exact inverse cell mass matrix.
#include "../../include/sipg.h"
#include "ctx.h"
#include "kernels.cuh"
#include "sweeps.cuh"

#include <chrono>
#include <cmath>

namespace sipg {
namespace {

using namespace sweeps;

template <int N>
__global__ void __launch_bounds__(kSplitThreads) pen_tau_kernel(LevelGeom g, SplitTab tab,
                                                                const double* __restrict__ u, double zeta_div,
                                                                double zeta_cont, double dt,
                                                                double* __restrict__ tdiv,
                                                                double* __restrict__ tcon) {
  constexpr int N3 = N * N * N;
  __shared__ STabSm T;
  __shared__ double U[3][N3], Q[3][N3], T0[N3], T1[N3];
  __shared__ double red[kSplitThreads];
  const int e = blockIdx.x;
  load_tab(tab, T);
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) U[i / N3][i % N3] = u[(size_t)e * 3 * N3 + i];
  __syncthreads();
  for (int c = 0; c < 3; ++c) sweep3<N, N, false>(T.S, N, U[c], T0, T1, Q[c]);
  const double vol = g.h[0] * g.h[1] * g.h[2];
  double acc = 0.0;
  for (int q = threadIdx.x; q < N3; q += blockDim.x)
    acc += cell_weight(T, q, N, vol) * sqrt(Q[0][q] * Q[0][q] + Q[1][q] * Q[1][q] + Q[2][q] * Q[2][q]);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double ubar = red[0] / vol;
    tdiv[e] = zeta_div * ubar * cbrt(vol) / (double)N * dt;
    tcon[e] = zeta_cont * ubar * dt;
  }
}

template <int N>
__global__ void __launch_bounds__(kSplitThreads) pen_apply_kernel(LevelGeom g, SplitTab tab,
                                                                  const double* __restrict__ tdiv,
                                                                  const double* __restrict__ tcon,
                                                                  const double* __restrict__ x,
                                                                  double* __restrict__ y) {
  constexpr int N3 = N * N * N, N2 = N * N;
  __shared__ STabSm T;
  __shared__ double X[3][N3], OUT[3][N3], Q[N3], DV[N3], T0[N3], T1[N3];
  __shared__ double FA[N2], FT[N2], FR[N2];
  const int e = blockIdx.x;
  load_tab(tab, T);
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) X[i / N3][i % N3] = x[(size_t)e * 3 * N3 + i];
  for (int i = threadIdx.x; i < N3; i += blockDim.x) DV[i] = 0.0;
  __syncthreads();
  const double detJ = g.h[0] * g.h[1] * g.h[2];
  // div x at the Gauss points
  for (int c = 0; c < 3; ++c) {
    sweep<N, N, N, 0, N, false>(c == 0 ? T.DS : T.S, N, X[c], T0);
    __syncthreads();
    sweep<N, N, N, 1, N, false>(c == 1 ? T.DS : T.S, N, T0, T1);
    __syncthreads();
    sweep<N, N, N, 2, N, false>(c == 2 ? T.DS : T.S, N, T1, Q);
    __syncthreads();
    for (int q = threadIdx.x; q < N3; q += blockDim.x) DV[q] += g.ih[c] * Q[q];
    __syncthreads();
  }
  const double td = tdiv[e];
  for (int q = threadIdx.x; q < N3; q += blockDim.x) DV[q] *= td * cell_weight(T, q, N, detJ);
  __syncthreads();
  for (int c = 0; c < 3; ++c) {
    // (phi_i, x_c): values at the Gauss points, weights, transposed sweeps
    sweep3<N, N, false>(T.S, N, X[c], T0, T1, Q);
    for (int q = threadIdx.x; q < N3; q += blockDim.x) Q[q] *= cell_weight(T, q, N, detJ);
    __syncthreads();
    sweep3<N, N, true>(T.S, N, Q, T0, T1, OUT[c]);
    // (d phi_i / d x_c, tau_div div x)
    sweep<N, N, N, 0, N, true>(c == 0 ? T.DS : T.S, N, DV, T0);
    __syncthreads();
    sweep<N, N, N, 1, N, true>(c == 1 ? T.DS : T.S, N, T0, T1);
    __syncthreads();
    sweep<N, N, N, 2, N, true>(c == 2 ? T.DS : T.S, N, T1, Q);
    __syncthreads();
    for (int i = threadIdx.x; i < N3; i += blockDim.x) OUT[c][i] += g.ih[c] * Q[i];
    __syncthreads();
  }
  const double tc = tcon[e];
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, s = f & 1;
    const int nb = cell_neighbor(g, e, f);
    if (nb < 0 && face_bc(g, e, f) != 0) continue;  // Neumann wall
    int t1, t2;
    face_dirs(d, &t1, &t2);
    const double tau = nb >= 0 ? 0.5 * (tc + tcon[nb]) : tc;
    for (int p = threadIdx.x; p < N2; p += blockDim.x) {
      const double out = nb >= 0 ? x[((size_t)nb * 3 + d) * N3 + fnode(d, 1 - s, p % N, p / N, N)] : 0.0;
      FA[p] = X[d][fnode(d, s, p % N, p / N, N)] - out;
    }
    __syncthreads();
    sweep<N, N, 1, 0, N, false>(T.S, N, FA, FT);
    __syncthreads();
    sweep<N, N, 1, 1, N, false>(T.S, N, FT, FR);
    __syncthreads();
    const double area = g.h[t1] * g.h[t2];
    for (int q = threadIdx.x; q < N2; q += blockDim.x) FR[q] *= tau * T.gw[q % N] * T.gw[q / N] * area;
    __syncthreads();
    sweep<N, N, 1, 0, N, true>(T.S, N, FR, FT);
    __syncthreads();
    sweep<N, N, 1, 1, N, true>(T.S, N, FT, FA);
    __syncthreads();
    for (int p = threadIdx.x; p < N2; p += blockDim.x) OUT[d][fnode(d, s, p % N, p / N, N)] += FA[p];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) y[(size_t)e * 3 * N3 + i] = OUT[i / N3][i % N3];
}

template <int N>
__global__ void __launch_bounds__(kSplitThreads) pen_wall_kernel(LevelGeom g, SplitTab tab, Wall wall,
                                                                 const double* __restrict__ tcon,
                                                                 double* __restrict__ y) {
  constexpr int N3 = N * N * N, N2 = N * N;
  __shared__ STabSm T;
  __shared__ double FA[N2], FT[N2], FR[N2];
  const int e = blockIdx.x;
  load_tab(tab, T);
  __syncthreads();
  for (int f = 0; f < 6; ++f) {
    if (cell_neighbor(g, e, f) >= 0 || face_bc(g, e, f) != 0) continue;
    const int d = f >> 1, s = f & 1;
    int t1, t2;
    face_dirs(d, &t1, &t2);
    const double c = tcon[e] * g.h[t1] * g.h[t2];
    for (int q = threadIdx.x; q < N2; q += blockDim.x)
      FA[q] = c * wall_val(wall, g, e, f, q, d, N2) * T.gw[q % N] * T.gw[q / N];
    __syncthreads();
    sweep<N, N, 1, 0, N, true>(T.S, N, FA, FT);
    __syncthreads();
    sweep<N, N, 1, 1, N, true>(T.S, N, FT, FR);
    __syncthreads();
    for (int p = threadIdx.x; p < N2; p += blockDim.x)
      y[((size_t)e * 3 + d) * N3 + fnode(d, s, p % N, p / N, N)] += FR[p];
    __syncthreads();
  }
}

}  // namespace

#define SIPG_PEN_DISPATCH(NN, CALL)                  \
  switch (NN) {                                       \
    case 3: { constexpr int N = 3; CALL; break; }     \
    case 4: { constexpr int N = 4; CALL; break; }     \
    case 5: { constexpr int N = 5; CALL; break; }     \
    case 6: { constexpr int N = 6; CALL; break; }     \
    default: return cudaErrorInvalidValue;            \
  }

cudaError_t launch_penalty_tau(int n, const LevelGeom& g, const SplitTab& tab, const double* u, double zeta_div,
                               double zeta_cont, double dt, double* tdiv, double* tcon, cudaStream_t st) {
  if (g.ncells == 0) return cudaSuccess;
  SIPG_PEN_DISPATCH(n, (pen_tau_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, u, zeta_div, zeta_cont, dt,
                                                                            tdiv, tcon)));
  return cudaGetLastError();
}

cudaError_t launch_penalty_apply(int n, const LevelGeom& g, const SplitTab& tab, const double* tdiv,
                                 const double* tcon, const double* x, double* y, cudaStream_t st) {
  if (g.ncells == 0) return cudaSuccess;
  SIPG_PEN_DISPATCH(n, (pen_apply_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, tdiv, tcon, x, y)));
  return cudaGetLastError();
}

cudaError_t launch_penalty_wall(int n, const LevelGeom& g, const SplitTab& tab, const WallArg& wall_g,
                                const double* tcon, double* y, cudaStream_t st) {
  if ((!wall_g.side && !wall_g.pts) || g.ncells == 0) return cudaSuccess;
  Wall w{};
  bool any = wall_g.pts != nullptr;
  for (int i = 0; i < 18; ++i) {
    w.g[i / 3][i % 3] = wall_g.side ? wall_g.side[i] : 0.0;
    any |= w.g[i / 3][i % 3] != 0.0;
  }
  w.pts = wall_g.pts;
  if (!any) return cudaSuccess;
  SIPG_PEN_DISPATCH(n, (pen_wall_kernel<N><<<g.ncells, kSplitThreads, 0, st>>>(g, tab, w, tcon, y)));
  return cudaGetLastError();
}

}  // namespace sipg

using namespace sipg;

#define CK(expr)                                                              \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess) return ctx->fail(SIPG_ERR_CUDA, #expr, e_);        \
  } while (0)

namespace {

int check_penalty(sipg_ctx* ctx) {
  if (ctx->opts.k_u < 2 || ctx->opts.k_u > 5) return ctx->fail(SIPG_ERR_INVALID, "velocity degree 2..5");
  if (ctx->mapped) return ctx->fail(SIPG_ERR_INVALID, "the penalty step is built for affine cells only");
  return SIPG_OK;
}

}  // namespace

int sipg_ctx::penalty_work() {
  sipg_ctx* ctx = this;
  const Level& L = hier[SIPG_OP_VISCOUS].L[0];
  if (pw.n == L.ndofs) return SIPG_OK;
  for (double* p : {pw.tdiv, pw.tcon, pw.b, pw.r, pw.z, pw.p, pw.q}) cudaFree(p);
  pw = PenaltyWork{};
  CK(cudaMalloc(&pw.tdiv, sizeof(double) * L.g.ncells));
  CK(cudaMalloc(&pw.tcon, sizeof(double) * L.g.ncells));
  for (double** v : {&pw.b, &pw.r, &pw.z, &pw.p, &pw.q}) CK(cudaMalloc(v, sizeof(double) * L.ndofs));
  pw.n = L.ndofs;
  return SIPG_OK;
}

int sipg_ctx::penalty_solve(const WallArg& wall_g, const double* u, double dt, double zeta_div, double zeta_cont,
                            double rtol, int maxit, double* x, int* iterations, double* rel_residual) {
  sipg_ctx* ctx = this;
  int rc = penalty_work();
  if (rc) return rc;
  const Level& L = hier[SIPG_OP_VISCOUS].L[0];
  const SplitTab& tab = stabs[L.n];
  const int64_t n = L.ndofs;
  CK(launch_penalty_tau(L.n, L.g, tab, u, zeta_div, zeta_cont, dt, pw.tdiv, pw.tcon, st));
  // b = M u + wall data; x0 = u (K is the mass matrix plus Courant-number-sized terms)
  if ((rc = mass_apply(SIPG_OP_VISCOUS, SIPG_F64_FF, u, pw.b, 1.0, false))) return rc;
  CK(launch_penalty_wall(L.n, L.g, tab, wall_g, pw.tcon, pw.b, st));
  if (x != u) CK(cudaMemcpyAsync(x, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  CK(launch_penalty_apply(L.n, L.g, tab, pw.tdiv, pw.tcon, x, pw.q, st));
  CK(launch_sub<double>(n, pw.b, pw.q, pw.r, st));
  double bb, rr;
  if ((rc = dot(n, pw.b, pw.b, &bb))) return rc;
  if ((rc = dot(n, pw.r, pw.r, &rr))) return rc;
  const double target = rtol * std::sqrt(bb);
  int it = 0, status = SIPG_OK;
  if (!std::isfinite(rr)) status = SIPG_ERR_NAN;
  if (status == SIPG_OK && std::sqrt(rr) > target) {
    if ((rc = mass_apply(SIPG_OP_VISCOUS, SIPG_F64_FF, pw.r, pw.z, 1.0, true))) return rc;
    CK(cudaMemcpyAsync(pw.p, pw.z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    double rz;
    if ((rc = dot(n, pw.r, pw.z, &rz))) return rc;
    while (true) {
      if (it >= maxit) { status = SIPG_ERR_MAXIT; break; }
      CK(launch_penalty_apply(L.n, L.g, tab, pw.tdiv, pw.tcon, pw.p, pw.q, st));
      double pq;
      if ((rc = dot(n, pw.p, pw.q, &pq))) return rc;
      if (!std::isfinite(pq)) { status = SIPG_ERR_NAN; break; }
      if (!(pq > 0)) { status = SIPG_ERR_BREAKDOWN; break; }
      const double alpha = rz / pq;
      CK(launch_add_scaled_f64(n, alpha, pw.p, x, st));
      CK(launch_add_scaled_f64(n, -alpha, pw.q, pw.r, st));
      ++it;
      if ((rc = dot(n, pw.r, pw.r, &rr))) return rc;
      if (!std::isfinite(rr)) { status = SIPG_ERR_NAN; break; }
      if (std::sqrt(rr) <= target) break;
      if ((rc = mass_apply(SIPG_OP_VISCOUS, SIPG_F64_FF, pw.r, pw.z, 1.0, true))) return rc;
      double rz_new;
      if ((rc = dot(n, pw.r, pw.z, &rz_new))) return rc;
      CK(launch_axpby<double>(n, 1.0, pw.z, rz_new / rz, pw.p, st));
      rz = rz_new;
    }
  }
  // true residual of the returned velocity
  CK(launch_penalty_apply(L.n, L.g, tab, pw.tdiv, pw.tcon, x, pw.q, st));
  CK(launch_sub<double>(n, pw.b, pw.q, pw.r, st));
  if ((rc = dot(n, pw.r, pw.r, &rr))) return rc;
  if (iterations) *iterations = it;
  if (rel_residual) *rel_residual = bb > 0 ? std::sqrt(rr / bb) : std::sqrt(rr);
  if (status == SIPG_ERR_MAXIT) return fail(status, "penalty step: iteration limit");
  if (status != SIPG_OK) return fail(status, "penalty step: CG breakdown");
  return SIPG_OK;
}

extern "C" int sipg_penalty_tau(sipg_ctx* ctx, const double* u, double dt, double zeta_div, double zeta_cont,
                                double* tau_div, double* tau_cont) {
  if (!ctx || !u || !tau_div || !tau_cont || !(dt > 0)) return SIPG_ERR_INVALID;
  int rc = check_penalty(ctx);
  if (rc) return rc;
  const Level& L = ctx->hier[SIPG_OP_VISCOUS].L[0];
  CK(launch_penalty_tau(L.n, L.g, ctx->stabs[L.n], u, zeta_div, zeta_cont, dt, tau_div, tau_cont, ctx->st));
  return SIPG_OK;
}

extern "C" int sipg_penalty_apply(sipg_ctx* ctx, const double* tau_div, const double* tau_cont, const double* x,
                                  double* y) {
  if (!ctx || !tau_div || !tau_cont || !x || !y || x == y) return SIPG_ERR_INVALID;
  int rc = check_penalty(ctx);
  if (rc) return rc;
  const Level& L = ctx->hier[SIPG_OP_VISCOUS].L[0];
  CK(launch_penalty_apply(L.n, L.g, ctx->stabs[L.n], tau_div, tau_cont, x, y, ctx->st));
  return SIPG_OK;
}

extern "C" int sipg_penalty_wall_rhs(sipg_ctx* ctx, const double* wall_g, const double* tau_cont, double* y) {
  if (!ctx || !tau_cont || !y) return SIPG_ERR_INVALID;
  int rc = check_penalty(ctx);
  if (rc) return rc;
  const Level& L = ctx->hier[SIPG_OP_VISCOUS].L[0];
  CK(cudaMemsetAsync(y, 0, sizeof(double) * L.ndofs, ctx->st));
  CK(launch_penalty_wall(L.n, L.g, ctx->stabs[L.n], wall_g, tau_cont, y, ctx->st));
  return SIPG_OK;
}

extern "C" int sipg_penalty_step(sipg_ctx* ctx, const double* wall_g, const double* u, double dt,
                                 double zeta_div, double zeta_cont, double rtol, int maxit, double* u_out,
                                 int* iterations, double* rel_residual) {
  if (!ctx || !u || !u_out || !(dt > 0) || !(rtol > 0) || maxit < 1) return SIPG_ERR_INVALID;
  int rc = check_penalty(ctx);
  if (rc) return rc;
  rc = ctx->penalty_solve(wall_g, u, dt, zeta_div, zeta_cont, rtol, maxit, u_out, iterations, rel_residual);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->st));
  return SIPG_OK;
}
