// One time step of the projection (dual splitting) scheme on affine grids (the
// box, the backward-facing-step channel) and on trilinear cells (the jittered
// channel), Sec. 3.2 / 5.1, Alg. 1, the convective term explicit (alpha_c = 0)
// or, on affine grids, linearly implicit in the viscous step (alpha_c = 1,
// u* = u#, GMRES): host sequence of library kernels (split.cu / mapped_split.cu
// forms, cell mass operators, MG-CG / GMRES solves, the Picard loop, the
// optional divergence and continuity penalty step on affine grids).
//
// State between steps: u^n, u^{n-1}, C(u^{n-1}) (the convective vector of the
// previous step is reused), p^n (initial guess of the next pressure solve).
#include "../../include/sipg.h"
#include "ctx.h"
#include "kernels.cuh"

#include <chrono>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

using namespace sipg;

#define CK(expr)                                                              \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess) return ctx->fail(SIPG_ERR_CUDA, #expr, e_);        \
  } while (0)

namespace {

using Clock = std::chrono::steady_clock;

double secs(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }

// every boundary id present: velocity Dirichlet + pressure Neumann (wall, inflow) or
// velocity Neumann + pressure Dirichlet (outflow)
bool walls_ok(const sipg_ctx* ctx) {
  const LevelGeom& gu = ctx->hier[SIPG_OP_VISCOUS].L[0].g;
  const LevelGeom& gp = ctx->hier[SIPG_OP_POISSON].L[0].g;
  for (int i = 0; i < 7; ++i) {
    if (!(ctx->used_ids >> i & 1)) continue;
    const bool wall = gu.bc[i] == SIPG_BC_DIRICHLET && gp.bc[i] == SIPG_BC_NEUMANN;
    const bool outflow = gu.bc[i] == SIPG_BC_NEUMANN && gp.bc[i] == SIPG_BC_DIRICHLET;
    if (!wall && !outflow) return false;
  }
  return true;
}

int check_forms(sipg_ctx* ctx) {
  if (ctx->opts.k_u < 2 || ctx->opts.k_u > 5) return ctx->fail(SIPG_ERR_INVALID, "velocity degree 2..5");
  return SIPG_OK;
}

// the forms of the fine velocity level, affine (split.cu) or trilinear (mapped_split.cu)
cudaError_t form_convective(sipg_ctx* ctx, const WallArg& w, const double* u, double* y) {
  const Level& L = ctx->hier[SIPG_OP_VISCOUS].L[0];
  return ctx->mapped ? launch_mapped_convective(L.n, L.g, ctx->stabs[L.n], L.verts, w, u, y, ctx->st)
                     : launch_convective(L.n, L.g, ctx->stabs[L.n], w, u, y, ctx->st);
}
cudaError_t form_projection(sipg_ctx* ctx, const double* p, double* y) {
  const Level& L = ctx->hier[SIPG_OP_VISCOUS].L[0];
  return ctx->mapped ? launch_mapped_projection_rhs(L.n, L.g, ctx->stabs[L.n], L.verts, p, y, ctx->st)
                     : launch_projection_rhs(L.n, L.g, ctx->stabs[L.n], p, y, ctx->st);
}
cudaError_t form_viscous_wall(sipg_ctx* ctx, const WallArg& w, double* y) {
  const Level& L = ctx->hier[SIPG_OP_VISCOUS].L[0];
  return ctx->mapped
             ? launch_mapped_viscous_wall_rhs(L.n, L.g, ctx->stabs[L.n], L.verts, L.lam, w, L.nu_face64, y, ctx->st)
             : launch_viscous_wall_rhs(L.n, L.g, ctx->stabs[L.n], w, L.nu_face64, y, ctx->st);
}

}  // namespace

extern "C" void sipg_default_step_opts(sipg_step_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->dt = 0.0;
  o->body = nullptr;
  o->viscosity_mode = SIPG_VISC_LINEAR_IMPLICIT;
  o->convective_mode = SIPG_CONV_EXPLICIT;
  o->gmres_restart = 30;
  o->ppe_rtol = 1e-8;
  o->visc_rtol = 1e-8;
  o->maxit = 1000;
  sipg_default_picard_opts(&o->picard);
  o->penalty = 0;
  o->penalty_rtol = 1e-10;
}

extern "C" int sipg_convective_apply(sipg_ctx* ctx, const double* wall_g, const double* u, double* y) {
  if (!ctx || !u || !y || u == y) return SIPG_ERR_INVALID;
  int rc = check_forms(ctx);
  if (rc) return rc;
  CK(form_convective(ctx, WallArg(wall_g), u, y));
  return SIPG_OK;
}

extern "C" int sipg_convective_lin_apply(sipg_ctx* ctx, const double* w, const double* wall_w, const double* wall_u,
                                         const double* u, double* y) {
  if (!ctx || !w || !u || !y || u == y || w == y) return SIPG_ERR_INVALID;
  int rc = check_forms(ctx);
  if (rc) return rc;
  if (ctx->mapped) return ctx->fail(SIPG_ERR_INVALID, "the linearised convective form is built for affine cells");
  const Level& L = ctx->hier[SIPG_OP_VISCOUS].L[0];
  CK(launch_convective_lin(L.n, L.g, ctx->stabs[L.n], wall_w, wall_u, w, u, y, ctx->st));
  return SIPG_OK;
}

extern "C" int sipg_projection_rhs(sipg_ctx* ctx, const double* p, double* y) {
  if (!ctx || !p || !y) return SIPG_ERR_INVALID;
  int rc = check_forms(ctx);
  if (rc) return rc;
  CK(form_projection(ctx, p, y));
  return SIPG_OK;
}

extern "C" int sipg_viscous_wall_rhs(sipg_ctx* ctx, const double* wall_g, double* y) {
  if (!ctx || !y) return SIPG_ERR_INVALID;
  int rc = check_forms(ctx);
  if (rc) return rc;
  if (!ctx->have_nu) return ctx->fail(SIPG_ERR_STATE, "set the viscosity first");
  CK(form_viscous_wall(ctx, WallArg(wall_g), y));
  return SIPG_OK;
}

extern "C" int sipg_cfl_dt(sipg_ctx* ctx, const double* u, double courant, double* dt) {
  if (!ctx || !u || !dt || !(courant > 0)) return SIPG_ERR_INVALID;
  int rc = check_forms(ctx);
  if (rc) return rc;
  auto& S = ctx->ss;
  if (!S.vmax) CK(cudaMalloc(&S.vmax, sizeof(unsigned long long)));
  const Level& L = ctx->hier[SIPG_OP_VISCOUS].L[0];
  if (ctx->mapped)
    CK(launch_mapped_cfl_max(L.n, L.g, ctx->stabs[L.n], L.verts, u, S.vmax, ctx->st));
  else
    CK(launch_cfl_max(L.n, L.g, ctx->stabs[L.n], u, S.vmax, ctx->st));
  unsigned long long bits = 0;
  CK(cudaMemcpyAsync(&bits, S.vmax, sizeof(bits), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  double vmax;
  std::memcpy(&vmax, &bits, sizeof(vmax));
  if (!(vmax > 0) || !std::isfinite(vmax)) return ctx->fail(SIPG_ERR_INVALID, "CFL time step of a zero velocity");
  *dt = courant / std::pow((double)L.k, 1.5) / vmax;
  return SIPG_OK;
}

extern "C" int sipg_boundary_faces(sipg_ctx* ctx, int* nbf, int* cell_face_id, double* xyz) {
  if (!ctx) return SIPG_ERR_INVALID;
  const Level& L = ctx->hier[SIPG_OP_VISCOUS].L[0];
  const LevelGeom& g = L.g;
  const int nb = n_wall_faces(g);
  if (nbf) *nbf = nb;
  if (cell_face_id) {
    if (g.nbr) {
      std::vector<int> bf(nb), nbr((size_t)g.ncells * 6);
      CK(cudaMemcpy(bf.data(), g.bface, sizeof(int) * nb, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(nbr.data(), g.nbr, sizeof(int) * nbr.size(), cudaMemcpyDeviceToHost));
      for (int b = 0; b < nb; ++b) {
        cell_face_id[3 * b + 0] = bf[b] / 6;
        cell_face_id[3 * b + 1] = bf[b] % 6;
        cell_face_id[3 * b + 2] = (-1 - nbr[bf[b]]) & 7;
      }
    } else {  // the plain box: side by side, each lexicographic over t1 < t2
      const int dims[3] = {g.nx, g.ny, g.nz};
      int b = 0;
      for (int f = 0; f < 6; ++f) {
        const int d = f >> 1, s = f & 1;
        const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        for (int j2 = 0; j2 < dims[t2]; ++j2)
          for (int j1 = 0; j1 < dims[t1]; ++j1, ++b) {
            int ijk[3];
            ijk[d] = s ? dims[d] - 1 : 0;
            ijk[t1] = j1;
            ijk[t2] = j2;
            cell_face_id[3 * b + 0] = (ijk[2] * g.ny + ijk[1]) * g.nx + ijk[0];
            cell_face_id[3 * b + 1] = f;
            cell_face_id[3 * b + 2] = f;
          }
      }
    }
  }
  if (xyz) {
    if (ctx->mapped)
      CK(launch_mapped_boundary_points(L.n, g, ctx->stabs[L.n], L.verts, xyz, ctx->st));
    else
      CK(launch_boundary_points(L.n, g, ctx->stabs[L.n], xyz, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  return SIPG_OK;
}

extern "C" int sipg_step_init(sipg_ctx* ctx, const double* u0, const double* p0) {
  if (!ctx || !u0) return SIPG_ERR_INVALID;
  int rc = check_forms(ctx);
  if (rc) return rc;
  if (!walls_ok(ctx))
    return ctx->fail(SIPG_ERR_INVALID,
                     "the splitting step needs velocity-Dirichlet / pressure-Neumann walls or "
                     "velocity-Neumann / pressure-Dirichlet outflow faces");
  auto& S = ctx->ss;
  const int64_t nu = ctx->hier[SIPG_OP_VISCOUS].L[0].ndofs;
  const int64_t np = ctx->hier[SIPG_OP_POISSON].L[0].ndofs;
  const Level& L = ctx->hier[SIPG_OP_VISCOUS].L[0];
  const int64_t nsb = (int64_t)n_wall_faces(L.g) * L.n * L.n;
  for (double** v : {&S.u[0], &S.u[1], &S.conv[0], &S.conv[1], &S.uhat, &S.uhh, &S.tmp, &S.usharp, &S.bv})
    if (!*v) CK(cudaMalloc(v, sizeof(double) * nu));
  if (!S.p) CK(cudaMalloc(&S.p, sizeof(double) * np));
  if (!S.prhs) CK(cudaMalloc(&S.prhs, sizeof(double) * np));
  if (!S.sb) CK(cudaMalloc(&S.sb, sizeof(double) * nsb));
  CK(cudaMemcpyAsync(S.u[0], u0, sizeof(double) * nu, cudaMemcpyDeviceToDevice, ctx->st));
  if (p0)
    CK(cudaMemcpyAsync(S.p, p0, sizeof(double) * np, cudaMemcpyDeviceToDevice, ctx->st));
  else
    CK(cudaMemsetAsync(S.p, 0, sizeof(double) * np, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  S.n_hist = 1;
  S.conv1 = false;
  S.steps = 0;
  return SIPG_OK;
}

extern "C" int sipg_step_field(sipg_ctx* ctx, int which, double* out) {
  if (!ctx || !out) return SIPG_ERR_INVALID;
  auto& S = ctx->ss;
  if (S.n_hist == 0) return ctx->fail(SIPG_ERR_STATE, "sipg_step_init first");
  const int64_t nu = ctx->hier[SIPG_OP_VISCOUS].L[0].ndofs;
  const int64_t np = ctx->hier[SIPG_OP_POISSON].L[0].ndofs;
  const double* src = nullptr;
  int64_t n = nu;
  switch (which) {
    case SIPG_FIELD_U: src = S.u[0]; break;
    case SIPG_FIELD_U_PREV:
      if (S.n_hist < 2) return ctx->fail(SIPG_ERR_STATE, "no previous velocity yet");
      src = S.u[1];
      break;
    case SIPG_FIELD_P: src = S.p; n = np; break;
    case SIPG_FIELD_UHAT: src = S.uhat; break;
    case SIPG_FIELD_UHATHAT: src = S.uhh; break;
    case SIPG_FIELD_PPE_RHS: src = S.prhs; n = np; break;
    default: return ctx->fail(SIPG_ERR_INVALID, "unknown field");
  }
  if ((which == SIPG_FIELD_UHAT || which == SIPG_FIELD_UHATHAT || which == SIPG_FIELD_PPE_RHS) && S.steps == 0)
    return ctx->fail(SIPG_ERR_STATE, "no step taken yet");
  CK(cudaMemcpyAsync(out, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return SIPG_OK;
}

extern "C" int sipg_step(sipg_ctx* ctx, const sipg_rheology* rh, const sipg_step_opts* so_in,
                         sipg_step_stats* stats) {
  if (!ctx || !rh) return SIPG_ERR_INVALID;
  auto& S = ctx->ss;
  if (S.n_hist == 0) return ctx->fail(SIPG_ERR_STATE, "sipg_step_init first");
  sipg_step_opts so;
  sipg_default_step_opts(&so);
  if (so_in) so = *so_in;
  if (!(so.dt > 0) || !std::isfinite(so.dt)) return ctx->fail(SIPG_ERR_INVALID, "time step must be positive");
  if (rh->law != SIPG_LAW_CONSTANT && rh->law != SIPG_LAW_CARREAU)
    return ctx->fail(SIPG_ERR_INVALID, "the splitting step takes a constant or Carreau-Yasuda viscosity");
  bool wall_moving = so.wall_points != nullptr;
  for (double v : so.wall_velocity) wall_moving |= v != 0.0;
  if (so.viscosity_mode == SIPG_VISC_IMPLICIT && wall_moving)
    return ctx->fail(SIPG_ERR_INVALID, "the implicit-viscosity step is built for zero wall velocity");
  if (so.viscosity_mode != SIPG_VISC_IMPLICIT && so.viscosity_mode != SIPG_VISC_LINEAR_IMPLICIT)
    return ctx->fail(SIPG_ERR_INVALID, "unknown viscosity mode");
  if (so.convective_mode != SIPG_CONV_EXPLICIT && so.convective_mode != SIPG_CONV_LINEAR_IMPLICIT)
    return ctx->fail(SIPG_ERR_INVALID, "unknown convective mode");
  if (so.convective_mode == SIPG_CONV_LINEAR_IMPLICIT && so.viscosity_mode != SIPG_VISC_LINEAR_IMPLICIT)
    return ctx->fail(SIPG_ERR_INVALID, "the linearly implicit convective step takes the linear-implicit viscosity");
  if (ctx->mapped && (so.convective_mode != SIPG_CONV_EXPLICIT || so.penalty))
    return ctx->fail(SIPG_ERR_INVALID,
                     "trilinear cells: explicit convective term, no penalty step (the linearised convective "
                     "form and the penalty forms are built for affine cells)");
  RheologyDev law;
  const double* u0 = S.u[0];
  int rc = ctx->parse_rheology(rh, u0, &law);
  if (rc) return rc;
  const auto t0 = Clock::now();
  cudaStream_t st = ctx->st;
  const Level& Lu = ctx->hier[SIPG_OP_VISCOUS].L[0];
  const SplitTab& tab = ctx->stabs[Lu.n];
  const int64_t nu = Lu.ndofs;
  const double dt = so.dt;
  const int m = S.n_hist >= 2 ? 2 : 1;
  const double gamma0 = m == 2 ? 1.5 : 1.0;
  const double alpha[2] = {m == 2 ? 2.0 : 1.0, m == 2 ? -0.5 : 0.0};
  const double beta[2] = {m == 2 ? 2.0 : 1.0, m == 2 ? -1.0 : 0.0};
  const int m_p = m - 1 < 2 ? m - 1 : 2;
  const double betabar[2] = {m_p >= 1 ? (m_p == 2 ? 2.0 : 1.0) : 0.0, m_p == 2 ? -1.0 : 0.0};
  // wall data at t_{n+1} (pressure datum, viscous and penalty steps) and at t_n (C(u^n))
  const WallArg wall(so.wall_velocity, so.wall_points);
  const WallArg wall_n(so.wall_velocity, so.wall_points_prev ? so.wall_points_prev : so.wall_points);

  // ---- 1 convective step: C(u^n) (C(u^{n-1}) kept from the previous step)
  std::swap(S.conv[0], S.conv[1]);
  S.conv1 = S.steps > 0;
  CK(form_convective(ctx, wall_n, S.u[0], S.conv[0]));
  if (m == 2 && !S.conv1) CK(form_convective(ctx, wall_n, S.u[1], S.conv[1]));
  // tmp = sum_i alpha_i/dt u^{n-i} + b ; bv = M tmp - sum_i beta_i C_i ; uhat = (gamma0/dt M)^-1 bv
  CK(launch_scale(nu, alpha[0] / dt, S.u[0], S.tmp, st));
  if (m == 2) CK(launch_add_scaled_f64(nu, alpha[1] / dt, S.u[1], S.tmp, st));
  if (so.body) CK(launch_add_scaled_f64(nu, 1.0, so.body, S.tmp, st));
  if ((rc = ctx->mass_apply(SIPG_OP_VISCOUS, SIPG_F64_FF, S.tmp, S.bv, 1.0, false))) return rc;
  CK(launch_add_scaled_f64(nu, -beta[0], S.conv[0], S.bv, st));
  if (m == 2) CK(launch_add_scaled_f64(nu, -beta[1], S.conv[1], S.bv, st));
  if ((rc = ctx->mass_apply(SIPG_OP_VISCOUS, SIPG_F64_FF, S.bv, S.uhat, gamma0 / dt, true))) return rc;
  CK(cudaStreamSynchronize(st));
  const auto t1 = Clock::now();

  // ---- 2 pressure step
  PpeBndArgs pa{};
  pa.n_hist = m;
  pa.wconv[0] = beta[0] - betabar[0];
  pa.wconv[1] = m == 2 ? beta[1] - betabar[1] : 0.0;
  pa.visc = m_p > 0 ? 1 : 0;
  pa.betabar[0] = betabar[0];
  pa.betabar[1] = betabar[1];
  pa.gn_coef = -gamma0 / dt;
  if (ctx->mapped) {
    CK(launch_mapped_ppe_boundary(Lu.n, Lu.g, tab, Lu.verts, wall, pa, law, S.u[0], m == 2 ? S.u[1] : S.u[0], S.sb,
                                  st));
    CK(launch_mapped_ppe_rhs(Lu.n, Lu.g, tab, Lu.verts, gamma0 / dt, S.uhat, S.sb, S.prhs, st));
  } else {
    CK(launch_ppe_boundary(Lu.n, Lu.g, tab, wall, pa, law, S.u[0], m == 2 ? S.u[1] : S.u[0], S.sb, st));
    CK(launch_ppe_rhs(Lu.n, Lu.g, tab, gamma0 / dt, S.uhat, S.sb, S.prhs, st));
  }
  sipg_solve_opts ps{so.ppe_rtol, 0.0, so.maxit, SIPG_PRECOND_MG, 0.0};
  sipg_solve_stats pst{};
  rc = ctx->solve(SIPG_OP_POISSON, S.prhs, S.p, &ps, &pst);
  if (rc != SIPG_OK) return rc;
  const auto t2 = Clock::now();

  // ---- 3 projection step: uhh = uhat + (gamma0/dt M)^-1 [(div v, p) - (v, {{p}} n)]
  CK(form_projection(ctx, S.p, S.tmp));
  if ((rc = ctx->mass_apply(SIPG_OP_VISCOUS, SIPG_F64_FF, S.tmp, S.uhh, gamma0 / dt, true))) return rc;
  CK(launch_add_scaled_f64(nu, 1.0, S.uhat, S.uhh, st));
  CK(cudaStreamSynchronize(st));
  const auto t3 = Clock::now();

  // ---- 4 viscous step
  const double mc = gamma0 / dt;
  CK(launch_scale(nu, beta[0], S.u[0], S.usharp, st));  // u# = sum beta_i u^{n-i}
  if (m == 2) CK(launch_add_scaled_f64(nu, beta[1], S.u[1], S.usharp, st));
  if ((rc = ctx->mass_apply(SIPG_OP_VISCOUS, SIPG_F64_FF, S.uhh, S.bv, mc, false))) return rc;
  int visc_its = 0, updates = 0;
  double visc_res = 0.0;
  // the new velocity goes to u[1] (u^{n-1} is no longer needed: C(u^{n-1}) and u# are formed)
  CK(cudaMemcpyAsync(S.u[1], S.usharp, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st));
  if (so.viscosity_mode == SIPG_VISC_LINEAR_IMPLICIT) {
    if ((rc = ctx->eval_viscosity(law, S.usharp))) return rc;
    if (wall_moving) {
      CK(form_viscous_wall(ctx, wall, S.tmp));
      CK(launch_add_scaled_f64(nu, 1.0, S.tmp, S.bv, st));
    }
    sipg_solve_opts vs{so.visc_rtol, 0.0, so.maxit, SIPG_PRECOND_MG, mc};
    sipg_solve_stats vst{};
    if (so.convective_mode == SIPG_CONV_LINEAR_IMPLICIT) {
      // alpha_c = 1: + sum_i beta_i C(u^{n-i}) on the right, c_h(v, u; u#) on the left;
      // the wall-data part of c_h(v, u; u#) is the form at u = 0 with u's wall data
      CK(launch_add_scaled_f64(nu, beta[0], S.conv[0], S.bv, st));
      if (m == 2) CK(launch_add_scaled_f64(nu, beta[1], S.conv[1], S.bv, st));
      if (wall_moving) {
        CK(cudaMemsetAsync(S.uhat, 0, sizeof(double) * nu, st));
        CK(launch_convective_lin(Lu.n, Lu.g, tab, wall, wall, S.usharp, S.uhat, S.tmp, st));
        CK(launch_add_scaled_f64(nu, -1.0, S.tmp, S.bv, st));
      }
      rc = ctx->gmres_solve(S.usharp, wall, S.bv, S.u[1], vs, so.gmres_restart, &vst);
    } else {
      rc = ctx->solve(SIPG_OP_VISCOUS, S.bv, S.u[1], &vs, &vst);
    }
    if (rc != SIPG_OK) return rc;
    visc_its = vst.iterations;
    visc_res = vst.rel_residual;
    updates = 1;
  } else {
    sipg_picard_opts po = so.picard;
    po.mass_coeff = mc;
    sipg_picard_stats pst2{};
    rc = sipg_picard_solve(ctx, rh, S.bv, S.u[1], &po, &pst2);
    if (rc != SIPG_OK) return rc;
    visc_its = pst2.lin_iterations;
    updates = pst2.iterations;
    visc_res = pst2.res0 > 0 ? pst2.res / pst2.res0 : 0.0;
  }
  CK(cudaStreamSynchronize(st));
  const auto t4 = Clock::now();
  // ---- 5 divergence and continuity penalty step (in place)
  int pen_its = 0;
  if (so.penalty) {
    double pres = 0.0;
    rc = ctx->penalty_solve(wall, S.u[1], dt, 1.0, 1.0, so.penalty_rtol, so.maxit, S.u[1], &pen_its, &pres);
    if (rc != SIPG_OK) return rc;
  }
  std::swap(S.u[0], S.u[1]);  // u^{n+1} -> u[0], u^n -> u[1]
  CK(cudaStreamSynchronize(st));
  const auto t5 = Clock::now();
  S.n_hist = 2;
  S.steps += 1;
  if (stats) {
    stats->order = m;
    stats->ppe_iterations = pst.iterations;
    stats->ppe_rel_residual = pst.rel_residual;
    stats->visc_iterations = visc_its;
    stats->visc_rel_residual = visc_res;
    stats->picard_updates = updates;
    stats->t_convective = secs(t0, t1);
    stats->t_pressure = secs(t1, t2);
    stats->t_projection = secs(t2, t3);
    stats->t_viscous = secs(t3, t4);
    stats->t_penalty = secs(t4, t5);
    stats->penalty_iterations = pen_its;
    stats->seconds = secs(t0, t5);
    stats->status = SIPG_OK;
  }
  return SIPG_OK;
}
