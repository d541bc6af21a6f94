// Nonlinear viscous step: Picard updates of the viscosity with Aitken
// relaxation (Sec. 5.4, Alg. 1 with the convective term explicit).
//
// Per update k: nu <- eta(gamma_dot(eps(u^k))) on every multigrid level
// (Eq. viscosity_pointwise, the same kernels as sipg_set_viscosity), the full
// nonlinear residual r_k = b - ((gamma_0/dt) M + A(nu)) u^k, the stopping test,
// then a CG solve of the viscous step linearised at u^k started from u^k, and
// the relaxed update u^{k+1} = u^k + omega_k (u_tilde - u^k) with
// omega_k = -omega_{k-1} r_{k-1}.(r_k - r_{k-1}) / ||r_k - r_{k-1}||^2 (Irons and
// Tuck's factor on the residual vectors, as the paper computes it from the full
// nonlinear residual). The multigrid hierarchy is set up again for each new
// viscosity inside the solve. Every vector operation runs in the library's
// kernels; the host holds the loop and the scalars of the deterministic dots.
#include "../../include/sipg.h"
#include "ctx.h"
#include "kernels.cuh"

#include <chrono>
#include <cmath>
#include <utility>

using namespace sipg;

#define CK(expr)                                                              \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess) return ctx->fail(SIPG_ERR_CUDA, #expr, e_);        \
  } while (0)

extern "C" void sipg_default_picard_opts(sipg_picard_opts* o) {
  if (!o) return;
  o->mass_coeff = 0.0;
  o->rtol = 1e-6;
  o->atol = 1e-12;
  o->maxit = 20;
  o->aitken = 1;
  o->omega_init = 1.0;
  o->lin_rtol = 1e-3;
  o->lin_atol = 0.0;
  o->lin_maxit = 500;
  o->precond = SIPG_PRECOND_MG;
}

extern "C" int sipg_picard_solve(sipg_ctx* ctx, const sipg_rheology* rh, const double* b, double* u,
                                 const sipg_picard_opts* po_in, sipg_picard_stats* stats) {
  if (!ctx || !rh || !b || !u || b == u) return SIPG_ERR_INVALID;
  sipg_picard_opts po;
  sipg_default_picard_opts(&po);
  if (po_in) po = *po_in;
  if (po.maxit < 0 || !(po.rtol >= 0) || !(po.atol >= 0) || !(po.lin_rtol >= 0) || !(po.lin_atol >= 0) ||
      po.lin_maxit < 0 || po.precond < 0 || po.precond > 2 || !(po.mass_coeff >= 0) || !std::isfinite(po.omega_init))
    return ctx->fail(SIPG_ERR_INVALID, "bad Picard options");
  RheologyDev law;
  int rc = ctx->parse_rheology(rh, u, &law);
  if (rc) return rc;
  Hier& H = ctx->hier[SIPG_OP_VISCOUS];
  if (H.singular && !(po.mass_coeff > 0))
    return ctx->fail(SIPG_ERR_INVALID, "all-Neumann viscous operator is singular (rigid modes): give a mass term");
  const int64_t n = H.L[0].ndofs;
  cudaStream_t st = ctx->st;
  for (double*& p : ctx->pic)
    if (!p) CK(cudaMalloc(&p, sizeof(double) * n));
  double *r = ctx->pic[0], *r_prev = ctx->pic[1], *u_old = ctx->pic[2], *dr = ctx->pic[3];
  const auto t0 = std::chrono::steady_clock::now();

  // r = b - (m M + A(nu(u))) u with the viscosity refreshed from u
  auto residual = [&](double* out, double* norm) -> int {
    int e = ctx->eval_viscosity(law, u);
    if (e) return e;
    if ((e = ctx->krylov_apply(SIPG_OP_VISCOUS, u, dr, po.mass_coeff))) return e;
    CK(launch_sub<double>(n, b, dr, out, st));
    double rr;
    if ((e = ctx->dot(n, out, out, &rr))) return e;
    *norm = std::sqrt(rr);
    return std::isfinite(rr) ? SIPG_OK : ctx->fail(SIPG_ERR_NAN, "nonlinear residual is not finite");
  };

  double res0 = 0.0, res = 0.0;
  if ((rc = residual(r, &res0))) return rc;
  res = res0;
  int hist_n = 0;
  auto record = [&](double v) {
    if (stats && stats->residuals && hist_n < stats->history_len) stats->residuals[hist_n] = v;
    ++hist_n;
  };
  record(res0);
  int k = 0, lin_its = 0;
  double omega = po.omega_init;
  bool have_prev = false;
  auto converged = [&]() { return res <= po.rtol * res0 || res <= po.atol; };
  while (k < po.maxit && !converged()) {
    CK(cudaMemcpyAsync(u_old, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    sipg_solve_opts so{0.0, std::max(po.lin_rtol * res, po.lin_atol), po.lin_maxit, po.precond, po.mass_coeff};
    sipg_solve_stats ss{};
    rc = ctx->solve(SIPG_OP_VISCOUS, b, u, &so, &ss);  // u <- u_tilde
    if (rc != SIPG_OK && rc != SIPG_ERR_MAXIT) return rc;
    lin_its += ss.iterations;
    if (po.aitken && have_prev) {
      CK(launch_sub<double>(n, r, r_prev, dr, st));
      double den, num;
      if ((rc = ctx->dot(n, dr, dr, &den))) return rc;
      if ((rc = ctx->dot(n, r_prev, dr, &num))) return rc;
      if (den > 0.0) omega = -omega * num / den;
    } else if (!po.aitken) {
      omega = 1.0;
    }
    if (stats && stats->omegas && k < stats->history_len) stats->omegas[k] = omega;
    // u = u_old + omega (u_tilde - u_old)
    CK(launch_axpby<double>(n, 1.0 - omega, u_old, omega, u, st));
    std::swap(r, r_prev);
    have_prev = true;
    if ((rc = residual(r, &res))) return rc;
    record(res);
    ++k;
  }
  CK(cudaStreamSynchronize(st));
  const int status = converged() ? SIPG_OK : SIPG_ERR_MAXIT;
  if (stats) {
    stats->iterations = k;
    stats->lin_iterations = lin_its;
    stats->res0 = res0;
    stats->res = res;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->status = status;
  }
  if (status != SIPG_OK) ctx->fail(status, "Picard iteration did not converge within maxit updates");
  return status;
}
