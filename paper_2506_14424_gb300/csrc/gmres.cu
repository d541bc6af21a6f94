// Restarted GMRES with right preconditioning for the viscous-step operator
// with the linearly implicit convective term (alpha_c = 1, u* = u#):
//     K x = ((mass M + A(nu)) + C(w)) x = b,
// C(w) the upwind convective form of Eq. (convective_term_weak) with the
// transport velocity w fixed. C makes K non-symmetric, so CG does not apply.
// Preconditioner: the hp-multigrid V-cycle of the symmetric part mass M + A
// (or Jacobi / none). Arnoldi with modified Gram-Schmidt on the library's
// deterministic dot products; the Hessenberg least-squares problem is solved
// with Givens rotations on the host (Saad, Iterative Methods for Sparse
// Linear Systems, Alg. 9.5). The reported residual is recomputed from x.
#include "../../include/sipg.h"
#include "ctx.h"
#include "kernels.cuh"

#include <chrono>
#include <cmath>
#include <vector>

using namespace sipg;

#define CK(expr)                                                              \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess) return ctx->fail(SIPG_ERR_CUDA, #expr, e_);        \
  } while (0)

// y = K x
int sipg_ctx::convective_apply_total(const double* w, const WallArg& wall_w, const double* x, double* y,
                                     double mass) {
  sipg_ctx* ctx = this;
  int rc = krylov_apply(SIPG_OP_VISCOUS, x, y, mass);
  if (rc) return rc;
  if (!w) return SIPG_OK;
  const Level& L = hier[SIPG_OP_VISCOUS].L[0];
  double* t = gm.tmp;
  CK(launch_convective_lin(L.n, L.g, stabs[L.n], wall_w, nullptr, w, x, t, st));
  CK(launch_add_scaled_f64(L.ndofs, 1.0, t, y, st));
  return SIPG_OK;
}

int sipg_ctx::gmres_solve(const double* w, const WallArg& wall_w, const double* b, double* x,
                          const sipg_solve_opts& so, int restart, sipg_solve_stats* stats) {
  sipg_ctx* ctx = this;
  Hier& H = hier[SIPG_OP_VISCOUS];
  const int64_t n = H.L[0].ndofs;
  if (restart < 1 || restart > 200) return fail(SIPG_ERR_INVALID, "GMRES restart length 1..200");
  if (so.precond != SIPG_PRECOND_NONE && (!H.ready || H.setup_mass != so.mass_coeff)) {
    int rc = setup_operator(SIPG_OP_VISCOUS, so.mass_coeff);
    if (rc) return rc;
  }
  // workspace (before the first apply: the convective term uses gm.tmp):
  // restart + 1 Krylov vectors, z, tmp, r
  if (gm.m < restart || gm.n != n) {
    for (double* p : gm.V) cudaFree(p);
    gm.V.clear();
    cudaFree(gm.z); cudaFree(gm.tmp); cudaFree(gm.r);
    gm.z = gm.tmp = gm.r = nullptr;
    gm.m = 0;
    gm.V.assign(restart + 1, nullptr);
    for (double*& p : gm.V) CK(cudaMalloc(&p, sizeof(double) * n));
    CK(cudaMalloc(&gm.z, sizeof(double) * n));
    CK(cudaMalloc(&gm.tmp, sizeof(double) * n));
    CK(cudaMalloc(&gm.r, sizeof(double) * n));
    gm.m = restart;
    gm.n = n;
  }
  const auto t0 = std::chrono::steady_clock::now();
  auto precond = [&](const double* in, double* out) -> int {
    if (so.precond == SIPG_PRECOND_NONE) {
      CK(cudaMemcpyAsync(out, in, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      return SIPG_OK;
    }
    return precondition(SIPG_OP_VISCOUS, so.precond, in, out, so.mass_coeff);
  };
  double bb;
  int rc = dot(n, b, b, &bb);
  if (rc) return rc;
  const double bnorm = std::sqrt(bb);
  const double target = std::max(so.rtol * bnorm, so.atol);
  int its = 0, status = SIPG_ERR_MAXIT;
  std::vector<double> Hm((restart + 1) * restart), cs(restart), sn(restart), gvec(restart + 1), yv(restart);
  while (true) {
    // r = b - K x
    if ((rc = convective_apply_total(w, wall_w, x, gm.r, so.mass_coeff))) return rc;
    CK(launch_sub<double>(n, b, gm.r, gm.V[0], st));
    double beta2;
    if ((rc = dot(n, gm.V[0], gm.V[0], &beta2))) return rc;
    const double beta = std::sqrt(beta2);
    if (!std::isfinite(beta)) { status = SIPG_ERR_NAN; break; }
    if (beta <= target) { status = SIPG_OK; break; }
    if (its >= so.maxit) break;
    CK(launch_scale(n, 1.0 / beta, gm.V[0], gm.V[0], st));
    std::fill(gvec.begin(), gvec.end(), 0.0);
    gvec[0] = beta;
    int j = 0;
    for (; j < restart && its < so.maxit; ++j) {
      if ((rc = precond(gm.V[j], gm.z))) return rc;
      if ((rc = convective_apply_total(w, wall_w, gm.z, gm.V[j + 1], so.mass_coeff))) return rc;
      for (int i = 0; i <= j; ++i) {
        double hij;
        if ((rc = dot(n, gm.V[i], gm.V[j + 1], &hij))) return rc;
        Hm[i * restart + j] = hij;
        CK(launch_add_scaled_f64(n, -hij, gm.V[i], gm.V[j + 1], st));
      }
      double h2;
      if ((rc = dot(n, gm.V[j + 1], gm.V[j + 1], &h2))) return rc;
      const double hn = std::sqrt(h2);
      if (!std::isfinite(hn)) return fail(SIPG_ERR_NAN, "GMRES: non-finite Arnoldi vector");
      Hm[(j + 1) * restart + j] = hn;
      if (hn > 0.0) CK(launch_scale(n, 1.0 / hn, gm.V[j + 1], gm.V[j + 1], st));
      // previous rotations on column j, then a new one that zeroes H[j+1][j]
      for (int i = 0; i < j; ++i) {
        const double a = Hm[i * restart + j], c = Hm[(i + 1) * restart + j];
        Hm[i * restart + j] = cs[i] * a + sn[i] * c;
        Hm[(i + 1) * restart + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = Hm[j * restart + j], c = Hm[(j + 1) * restart + j];
      const double r = std::hypot(a, c);
      cs[j] = r > 0 ? a / r : 1.0;
      sn[j] = r > 0 ? c / r : 0.0;
      Hm[j * restart + j] = r;
      Hm[(j + 1) * restart + j] = 0.0;
      gvec[j + 1] = -sn[j] * gvec[j];
      gvec[j] = cs[j] * gvec[j];
      ++its;
      if (std::fabs(gvec[j + 1]) <= target || hn == 0.0) {
        ++j;
        break;
      }
    }
    // y = H^-1 g (upper triangular j x j), x += M^-1 (V y)
    for (int i = j - 1; i >= 0; --i) {
      double s = gvec[i];
      for (int k = i + 1; k < j; ++k) s -= Hm[i * restart + k] * yv[k];
      yv[i] = s / Hm[i * restart + i];
    }
    CK(launch_fill<double>(n, 0.0, gm.tmp, st));
    for (int i = 0; i < j; ++i) CK(launch_add_scaled_f64(n, yv[i], gm.V[i], gm.tmp, st));
    if ((rc = precond(gm.tmp, gm.z))) return rc;
    CK(launch_add_scaled_f64(n, 1.0, gm.z, x, st));
    // the recursive residual estimate can run ahead of the true one: the next
    // pass recomputes r = b - K x and either stops or restarts from it
  }
  // true residual of the returned iterate
  if ((rc = convective_apply_total(w, wall_w, x, gm.r, so.mass_coeff))) return rc;
  CK(launch_sub<double>(n, b, gm.r, gm.z, st));
  double rr;
  if ((rc = dot(n, gm.z, gm.z, &rr))) return rc;
  CK(cudaStreamSynchronize(st));
  if (stats) {
    stats->iterations = its;
    stats->rel_residual = bnorm > 0 ? std::sqrt(rr) / bnorm : std::sqrt(rr);
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->status = status;
  }
  if (status != SIPG_OK) return fail(status, "GMRES stopped before reaching the tolerance");
  return SIPG_OK;
}

extern "C" int sipg_solve_convective(sipg_ctx* ctx, const double* w, const double* wall_w, const double* b,
                                     double* x, const sipg_solve_opts* so_in, int restart,
                                     sipg_solve_stats* stats) {
  if (!ctx || !b || !x || b == x) return SIPG_ERR_INVALID;
  if (!ctx->have_nu) return ctx->fail(SIPG_ERR_STATE, "set the viscosity first");
  if (ctx->opts.k_u < 2 || ctx->opts.k_u > 5) return ctx->fail(SIPG_ERR_INVALID, "velocity degree 2..5");
  if (ctx->mapped && w) return ctx->fail(SIPG_ERR_INVALID, "the convective form is built for the box only");
  sipg_solve_opts so{1e-8, 0.0, 500, SIPG_PRECOND_MG, 0.0};
  if (so_in) so = *so_in;
  if (so.maxit < 0 || !(so.rtol >= 0) || so.precond < 0 || so.precond > 2)
    return ctx->fail(SIPG_ERR_INVALID, "bad solve options");
  if (ctx->hier[SIPG_OP_VISCOUS].singular && !(so.mass_coeff > 0))
    return ctx->fail(SIPG_ERR_INVALID, "all-Neumann viscous operator is singular (rigid modes): give a mass term");
  return ctx->gmres_solve(w, wall_w, b, x, so, restart, stats);
}
