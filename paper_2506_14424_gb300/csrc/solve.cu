// Preconditioned CG (FP64) and the hp-multigrid V-cycle (FP32 or FP64 inside),
// Sec. 5.4 of the paper:
//  * CG for the symmetric viscous and pressure systems;
//  * V-cycle over p-levels k -> 2 -> 1 and h-levels of the refined coarse
//    grid; Chebyshev-accelerated Jacobi smoothing (degree d, interval
//    [lmax/range, lmax], lmax = factor * Lanczos estimate, the textbook
//    three-term recurrence), one pre- and one post-smoothing application;
//  * transfers: prolongation = embedding, restriction = its transpose;
//  * coarsest level: FP64 direct solve (precomputed dense inverse) in both
//    precision modes.
#include "../../include/sipg.h"
#include "ctx.h"
#include "kernels.cuh"

#include <chrono>
#include <cmath>
#include <cstring>

using namespace sipg;

#define CK(expr)                                                              \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess) return ctx->fail(SIPG_ERR_CUDA, #expr, e_);        \
  } while (0)

namespace {
template <typename T> constexpr int prec_index() { return sizeof(T) == 8 ? 0 : 1; }
}  // namespace

template <typename T>
int sipg_ctx::transfer(int op, int l, int dir, const T* in, T* out) {
  sipg_ctx* ctx = this;
  const Hier& H = hier[op];
  const Level& F = H.L[l];
  const Level& C = H.L[l + 1];
  constexpr int pr = sizeof(T) == 8 ? 0 : 1;
  if (F.next_kind == 3) {  // DG level 0 -> continuous level of the same mesh and degree: P / P^T
    CK(launch_cg_map<T>(dir > 0 ? CG_GATHER : CG_SCATTER_SUM, C.cgg, in, out, 1, st));
    return SIPG_OK;
  }
  if (F.cg) {
    // continuous -> continuous: prolongation R_f Pdg P_c, restriction its transpose
    T* tf = static_cast<T*>(F.tdg[pr][0]);
    T* tc = static_cast<T*>(C.tdg[pr][0]);
    if (dir > 0) {
      CK(launch_cg_map<T>(CG_GATHER, C.cgg, in, tc, 1, st));
      if (F.next_kind == 1)
        CK(launch_p_transfer<T>(F.n, C.n, H.ncomp, F.g.ncells, F.tt, dir, tc, tf, st));
      else
        CK(launch_h_transfer<T>(F.n, H.ncomp, F.g, C.g, F.tt, dir, tc, tf, st));
      CK(launch_cg_map<T>(CG_PICK, F.cgg, tf, out, 1, st));
    } else {
      CK(launch_cg_map<T>(CG_PICK_T, F.cgg, in, tf, 1, st));
      if (F.next_kind == 1)
        CK(launch_p_transfer<T>(F.n, C.n, H.ncomp, F.g.ncells, F.tt, dir, tf, tc, st));
      else
        CK(launch_h_transfer<T>(F.n, H.ncomp, F.g, C.g, F.tt, dir, tf, tc, st));
      CK(launch_cg_map<T>(CG_SCATTER_SUM, C.cgg, tc, out, 1, st));
    }
    return SIPG_OK;
  }
  if (F.next_kind == 1)
    CK(launch_p_transfer<T>(F.n, C.n, H.ncomp, F.g.ncells, F.tt, dir, in, out, st));
  else
    CK(launch_h_transfer<T>(F.n, H.ncomp, F.g, C.g, F.tt, dir, in, out, st));
  return SIPG_OK;
}

// Chebyshev-Jacobi on level l: x <- S(x, b) with b = w[.][0], x = w[.][1],
// scratch t = w[.][2], d = w[.][3].
template <typename T>
int sipg_ctx::smooth(int op, int l, bool x_zero, double mass) {
  sipg_ctx* ctx = this;
  Level& L = hier[op].L[l];
  constexpr int p = prec_index<T>();
  T* b = (T*)L.w[p][0];
  T* x = (T*)L.w[p][1];
  T* t = (T*)L.w[p][2];
  T* d = (T*)L.w[p][3];
  const T* dinv = p == 0 ? (const T*)L.dinv64 : (const T*)L.dinv32;
  const double lmax = opts.cheb_lmax_factor * L.lmax;
  const double lmin = lmax / opts.cheb_range;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rho_old = 1.0 / sigma;
  const int64_t n = L.ndofs;
  if (x_zero) {
    CK(launch_cheb<T>(n, T(0), T(1.0 / theta), dinv, b, nullptr, d, x, true, st));
  } else {
    int rc = level_apply<T>(op, l, x, t, mass);
    if (rc) return rc;
    CK(launch_cheb<T>(n, T(0), T(1.0 / theta), dinv, b, t, d, x, false, st));
  }
  for (int it = 1; it < opts.cheb_degree; ++it) {
    const double rho = 1.0 / (2.0 * sigma - rho_old);
    int rc = level_apply<T>(op, l, x, t, mass);
    if (rc) return rc;
    CK(launch_cheb<T>(n, T(rho * rho_old), T(2.0 * rho / delta), dinv, b, t, d, x, false, st));
    rho_old = rho;
  }
  return SIPG_OK;
}

int sipg_ctx::coarse_solve64(int op) {
  sipg_ctx* ctx = this;
  Level& C = hier[op].L.back();
  CK(launch_gemv(C.N, C.Ainv, (const double*)C.w[0][0], (double*)C.w[0][1], st));
  return SIPG_OK;
}

// x_l = V(b_l) with b_l = w[.][0], result in w[.][1].
template <typename T>
int sipg_ctx::vcycle(int op, int l, double mass) {
  sipg_ctx* ctx = this;
  Hier& H = hier[op];
  Level& L = H.L[l];
  constexpr int p = prec_index<T>();
  if (l + 1 == (int)H.L.size()) {
    if (p == 1) CK((launch_cast<float, double>(L.ndofs, (const float*)L.w[1][0], (double*)L.w[0][0], st)));
    int rc = coarse_solve64(op);
    if (rc) return rc;
    if (p == 1) CK((launch_cast<double, float>(L.ndofs, (const double*)L.w[0][1], (float*)L.w[1][1], st)));
    return SIPG_OK;
  }
  int rc = smooth<T>(op, l, true, mass);
  if (rc) return rc;
  T* b = (T*)L.w[p][0];
  T* x = (T*)L.w[p][1];
  T* t = (T*)L.w[p][2];
  rc = level_apply<T>(op, l, x, t, mass);
  if (rc) return rc;
  CK(launch_sub<T>(L.ndofs, b, t, t, st));  // t = residual
  Level& C = H.L[l + 1];
  rc = transfer<T>(op, l, -1, t, (T*)C.w[p][0]);
  if (rc) return rc;
  rc = vcycle<T>(op, l + 1, mass);
  if (rc) return rc;
  rc = transfer<T>(op, l, +1, (const T*)C.w[p][1], t);
  if (rc) return rc;
  CK(launch_axpby<T>(L.ndofs, T(1), t, T(1), x, st));
  return smooth<T>(op, l, false, mass);
}

int sipg_ctx::precondition(int op, int kind, const double* r, double* z, double mass) {
  sipg_ctx* ctx = this;
  Hier& H = hier[op];
  Level& L0 = H.L[0];
  const int64_t n = L0.ndofs;
  if (kind == SIPG_PRECOND_NONE) {
    CK(cudaMemcpyAsync(z, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  } else if (kind == SIPG_PRECOND_JACOBI) {
    CK(launch_mul(n, L0.dinv64, r, z, st));
  } else {
    int rc;
    if (opts.mg_precision == SIPG_F32) {
      CK((launch_cast<double, float>(n, r, (float*)L0.w[1][0], st)));
      rc = vcycle<float>(op, 0, mass);
      if (rc) return rc;
      CK((launch_cast<float, double>(n, (const float*)L0.w[1][1], z, st)));
    } else {
      CK(cudaMemcpyAsync(L0.w[0][0], r, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      rc = vcycle<double>(op, 0, mass);
      if (rc) return rc;
      CK(cudaMemcpyAsync(z, L0.w[0][1], sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    }
  }
  if (H.singular && op == SIPG_OP_POISSON) return project_mean(n, z);
  return SIPG_OK;
}

int sipg_ctx::solve(int op, const double* b, double* x, const sipg_solve_opts* so_in, sipg_solve_stats* stats) {
  sipg_ctx* ctx = this;
  sipg_solve_opts so{1e-8, 0.0, 500, SIPG_PRECOND_MG, 0.0};
  if (so_in) so = *so_in;
  Hier& H = hier[op];
  if (H.singular && !(so.mass_coeff > 0) && op == SIPG_OP_VISCOUS)
    return fail(SIPG_ERR_INVALID, "all-Neumann viscous operator is singular (rigid modes): give a mass term");
  if (so.precond != SIPG_PRECOND_NONE && (!H.ready || H.setup_mass != so.mass_coeff)) {
    int rc = setup_operator(op, so.mass_coeff);
    if (rc) return rc;
  }
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = H.L[0].ndofs;
  double *r = H.cg[0], *z = H.cg[1], *p = H.cg[2], *q = H.cg[3], *bb = H.cg[4];
  const bool proj = H.singular && op == SIPG_OP_POISSON;
  CK(cudaMemcpyAsync(bb, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  if (proj) { int rc = project_mean(n, bb); if (rc) return rc; }
  int rc = krylov_apply(op, x, q, so.mass_coeff);
  if (rc) return rc;
  CK(launch_sub<double>(n, bb, q, r, st));
  if (proj) { rc = project_mean(n, r); if (rc) return rc; }
  double bnorm2, rr;
  if ((rc = dot(n, bb, bb, &bnorm2))) return rc;
  if ((rc = dot(n, r, r, &rr))) return rc;
  const double bnorm = std::sqrt(bnorm2);
  const double target = std::max(so.rtol * bnorm, so.atol);
  int status = SIPG_OK, it = 0, replacements = 0;
  constexpr int kMaxReplacements = 3;
  bool true_rr = false;  // r and rr hold the true residual of x
  if (!std::isfinite(rr)) status = SIPG_ERR_NAN;
  if (status == SIPG_OK && std::sqrt(rr) > target) {
    if ((rc = precondition(op, so.precond, r, z, so.mass_coeff))) return rc;
    CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    double rz;
    if ((rc = dot(n, r, z, &rz))) return rc;
    while (true) {
      if (it >= so.maxit) { status = SIPG_ERR_MAXIT; break; }
      if ((rc = krylov_apply(op, p, q, so.mass_coeff))) return rc;
      double pq;
      if ((rc = dot(n, p, q, &pq))) return rc;
      if (!std::isfinite(pq)) { status = SIPG_ERR_NAN; break; }
      if (!(pq > 0)) { status = SIPG_ERR_BREAKDOWN; break; }
      const double alpha = rz / pq;
      CK(launch_add_scaled_f64(n, alpha, p, x, st));
      CK(launch_add_scaled_f64(n, -alpha, q, r, st));
      if (proj) { if ((rc = project_mean(n, r))) return rc; }
      ++it;
      if ((rc = dot(n, r, r, &rr))) return rc;
      if (!std::isfinite(rr)) { status = SIPG_ERR_NAN; break; }
      if (std::sqrt(rr) <= target) {
        // confirm with the true residual b - A x: on large, high-contrast systems
        // rounding in the recursion can leave it a few times above the recursive
        // one; then restart from it (at most kMaxReplacements times, within maxit)
        if (replacements >= kMaxReplacements || it >= so.maxit) break;
        if ((rc = krylov_apply(op, x, q, so.mass_coeff))) return rc;
        CK(launch_sub<double>(n, bb, q, r, st));
        if (proj) { if ((rc = project_mean(n, r))) return rc; }
        if ((rc = dot(n, r, r, &rr))) return rc;
        true_rr = true;
        if (std::sqrt(rr) <= target) break;
        true_rr = false;
        ++replacements;
        if ((rc = precondition(op, so.precond, r, z, so.mass_coeff))) return rc;
        CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        if ((rc = dot(n, r, z, &rz))) return rc;
        continue;
      }
      if ((rc = precondition(op, so.precond, r, z, so.mass_coeff))) return rc;
      double rz_new;
      if ((rc = dot(n, r, z, &rz_new))) return rc;
      if (!std::isfinite(rz_new)) { status = SIPG_ERR_NAN; break; }
      CK(launch_axpby<double>(n, 1.0, z, rz_new / rz, p, st));
      rz = rz_new;
    }
  }
  // true residual of the returned iterate (already at hand after a confirmed convergence)
  if (!true_rr) {
    if ((rc = krylov_apply(op, x, q, so.mass_coeff))) return rc;
    CK(launch_sub<double>(n, bb, q, r, st));
    if (proj) { if ((rc = project_mean(n, r))) return rc; }
    if ((rc = dot(n, r, r, &rr))) return rc;
  }
  CK(cudaStreamSynchronize(st));
  const auto t1 = std::chrono::steady_clock::now();
  if (stats) {
    stats->iterations = it;
    stats->rel_residual = bnorm > 0 ? std::sqrt(rr) / bnorm : std::sqrt(rr);
    stats->seconds = std::chrono::duration<double>(t1 - t0).count();
    stats->status = status;
  }
  if (status != SIPG_OK) {
    char buf[128];
    snprintf(buf, sizeof buf, "solve stopped with status %d after %d iterations", status, it);
    err = buf;
  }
  return status;
}

// ---------------------------------------------------------------- C ABI
extern "C" int sipg_solve(sipg_ctx* ctx, int op, const double* b, double* x, const sipg_solve_opts* so,
                          sipg_solve_stats* stats) {
  if (!ctx || !b || !x || b == x) return SIPG_ERR_INVALID;
  if (op != SIPG_OP_VISCOUS && op != SIPG_OP_POISSON) return ctx->fail(SIPG_ERR_INVALID, "unknown operator");
  if (op == SIPG_OP_VISCOUS && !ctx->have_nu) return ctx->fail(SIPG_ERR_STATE, "set the viscosity first");
  if (so && (so->maxit < 0 || !(so->rtol >= 0) || so->precond < 0 || so->precond > 2))
    return ctx->fail(SIPG_ERR_INVALID, "bad solve options");
  return ctx->solve(op, b, x, so, stats);
}

extern "C" int sipg_get_viscosity(const sipg_ctx* cctx, int level, double* nu_cell, double* nu_face) {
  sipg_ctx* ctx = const_cast<sipg_ctx*>(cctx);
  if (!ctx || !ctx->have_nu) return SIPG_ERR_STATE;
  const Hier& H = ctx->hier[SIPG_OP_VISCOUS];
  if (level < 0 || level >= (int)H.L.size()) return SIPG_ERR_INVALID;
  const Level& L = H.L[level];
  const int64_t n3 = (int64_t)L.n * L.n * L.n, n2 = (int64_t)L.n * L.n;
  if (nu_cell)
    CK(cudaMemcpyAsync(nu_cell, L.nu_cell64, sizeof(double) * L.g.ncells * n3, cudaMemcpyDeviceToDevice, ctx->st));
  if (nu_face)
    CK(cudaMemcpyAsync(nu_face, L.nu_face64, sizeof(double) * L.g.ncells * 6 * n2, cudaMemcpyDeviceToDevice,
                       ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return SIPG_OK;
}

static int check_level(sipg_ctx* ctx, int op, int level) {
  if (op != SIPG_OP_VISCOUS && op != SIPG_OP_POISSON) return ctx->fail(SIPG_ERR_INVALID, "unknown operator");
  if (op == SIPG_OP_VISCOUS && !ctx->have_nu) return ctx->fail(SIPG_ERR_STATE, "set the viscosity first");
  if (level < 0 || level >= (int)ctx->hier[op].L.size()) return ctx->fail(SIPG_ERR_INVALID, "bad level");
  return ctx->ensure_setup(op);  // multigrid data of this operator
}

extern "C" int sipg_get_inverse_diagonal(const sipg_ctx* cctx, int op, int level, double* out) {
  sipg_ctx* ctx = const_cast<sipg_ctx*>(cctx);
  if (!ctx || !out) return SIPG_ERR_INVALID;
  int rc = check_level(ctx, op, level);
  if (rc) return rc;
  const Level& L = ctx->hier[op].L[level];
  CK(cudaMemcpyAsync(out, L.dinv64, sizeof(double) * L.ndofs, cudaMemcpyDeviceToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return SIPG_OK;
}

extern "C" int sipg_get_lmax_estimate(const sipg_ctx* cctx, int op, int level, double* lmax) {
  sipg_ctx* ctx = const_cast<sipg_ctx*>(cctx);
  if (!ctx || !lmax) return SIPG_ERR_INVALID;
  int rc = check_level(ctx, op, level);
  if (rc) return rc;
  *lmax = ctx->hier[op].L[level].lmax;
  return SIPG_OK;
}

extern "C" int sipg_transfer(sipg_ctx* ctx, int op, int level, int dir, int prec, const void* in, void* out) {
  if (!ctx || !in || !out || in == out) return SIPG_ERR_INVALID;
  int rc = check_level(ctx, op, level);
  if (rc) return rc;
  if (level + 1 >= (int)ctx->hier[op].L.size() || (dir != 1 && dir != -1))
    return ctx->fail(SIPG_ERR_INVALID, "no coarser level or bad direction");
  if (prec == SIPG_F64) return ctx->transfer<double>(op, level, dir, (const double*)in, (double*)out);
  if (prec == SIPG_F32) return ctx->transfer<float>(op, level, dir, (const float*)in, (float*)out);
  return ctx->fail(SIPG_ERR_INVALID, "bad precision");
}

extern "C" int sipg_smooth(sipg_ctx* ctx, int op, int level, int prec, const void* b, void* x) {
  if (!ctx || !b || !x) return SIPG_ERR_INVALID;
  int rc = check_level(ctx, op, level);
  if (rc) return rc;
  Level& L = ctx->hier[op].L[level];
  if (level + 1 == (int)ctx->hier[op].L.size()) return ctx->fail(SIPG_ERR_INVALID, "coarsest level has no smoother");
  const int p = prec == SIPG_F64 ? 0 : 1;
  if (prec != SIPG_F64 && prec != SIPG_F32) return ctx->fail(SIPG_ERR_INVALID, "bad precision");
  const size_t bytes = (p == 0 ? 8 : 4) * (size_t)L.ndofs;
  CK(cudaMemcpyAsync(L.w[p][0], b, bytes, cudaMemcpyDeviceToDevice, ctx->st));
  CK(cudaMemcpyAsync(L.w[p][1], x, bytes, cudaMemcpyDeviceToDevice, ctx->st));
  const double mass = ctx->hier[op].setup_mass;
  rc = p == 0 ? ctx->smooth<double>(op, level, false, mass) : ctx->smooth<float>(op, level, false, mass);
  if (rc) return rc;
  CK(cudaMemcpyAsync(x, L.w[p][1], bytes, cudaMemcpyDeviceToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return SIPG_OK;
}

extern "C" int sipg_vcycle(sipg_ctx* ctx, int op, const double* b, double* x) {
  if (!ctx || !b || !x || b == x) return SIPG_ERR_INVALID;
  int rc = check_level(ctx, op, 0);
  if (rc) return rc;
  rc = ctx->precondition(op, SIPG_PRECOND_MG, b, x, ctx->hier[op].setup_mass);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->st));
  return SIPG_OK;
}

extern "C" int sipg_node_points(const sipg_ctx* cctx, int op, int level, double* xyz_host) {
  sipg_ctx* ctx = const_cast<sipg_ctx*>(cctx);
  if (!ctx || !xyz_host || (op != 0 && op != 1)) return SIPG_ERR_INVALID;
  if (ctx->mapped) return ctx->fail(SIPG_ERR_INVALID, "node points of trilinear cells: map the reference nodes on the host");
  const Hier& H = ctx->hier[op];
  if (level < 0 || level >= (int)H.L.size()) return SIPG_ERR_INVALID;
  const Level& L = H.L[level];
  if (L.cg) return ctx->fail(SIPG_ERR_INVALID, "node points of a continuous level: the global Gauss-Lobatto grid");
  const int64_t total = (int64_t)L.g.ncells * L.n * L.n * L.n * 3;
  double* d = nullptr;
  CK(cudaMalloc(&d, sizeof(double) * total));
  cudaError_t e = launch_node_points(L.n, L.g, ctx->tabs[L.n], d, ctx->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(xyz_host, d, sizeof(double) * total, cudaMemcpyDeviceToHost, ctx->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  cudaFree(d);
  if (e != cudaSuccess) return ctx->fail(SIPG_ERR_CUDA, "node points", e);
  return SIPG_OK;
}

template int sipg_ctx::smooth<double>(int, int, bool, double);
template int sipg_ctx::smooth<float>(int, int, bool, double);
template int sipg_ctx::vcycle<double>(int, int, double);
template int sipg_ctx::vcycle<float>(int, int, double);
