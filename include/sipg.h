/*
 * sipg.h - C ABI of libsipg, a GB300 (sm_103a) implementation of the
 * matrix-free SIPG discontinuous Galerkin operators of arXiv 2506.14424
 * ("Higher-order discontinuous Galerkin splitting schemes for fluids with
 * variable viscosity") and of the CG / hp-multigrid solver around them.
 *
 * Conventions
 *  - Every call returns int: SIPG_OK (0), SIPG_PENDING (1) or a negative
 *    SIPG_ERR_* code. sipg_last_error() returns the message of the last
 *    failing call on a context. No C++ exception crosses this boundary.
 *  - "device" pointers are CUDA global-memory pointers of the current device
 *    (for example torch.empty(..., device='cuda').data_ptr()); "host"
 *    pointers are ordinary CPU memory. The caller owns every buffer passed
 *    in; the library owns the context, the mesh hierarchy, the viscosity
 *    storage, the multigrid levels and its workspaces. Nothing is freed
 *    across the boundary.
 *  - All work is ordered on the stream given to sipg_create (a cudaStream_t
 *    passed as void*, 0 = legacy default stream). Calls marked (sync) block
 *    until their work is done; the others are asynchronous.
 *  - Vector layout (shared with every test): DoF index
 *      ((cell * ncomp + c) * n + iz) * n * n + iy * n + ix,  n = k + 1,
 *    cells lexicographic with x fastest, nodes = k+1 Gauss-Lobatto points per
 *    direction on each cell. ncomp = 3 for velocity, 1 for pressure.
 *  - Quadrature: k+1 Gauss-Legendre points per direction in cells and on
 *    faces (Sec. 5 of the paper: as many quadrature as support points).
 */
#ifndef SIPG_H
#define SIPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
  SIPG_OK = 0,
  SIPG_PENDING = 1,
  SIPG_ERR_INVALID = -1,   /* bad argument, size or option */
  SIPG_ERR_CUDA = -2,      /* a CUDA runtime call failed */
  SIPG_ERR_NOMEM = -3,     /* allocation or HBM budget exceeded */
  SIPG_ERR_MAXIT = -4,     /* solver hit its iteration limit */
  SIPG_ERR_BREAKDOWN = -5, /* CG breakdown: p^T A p <= 0 */
  SIPG_ERR_NAN = -6,       /* NaN or Inf met in a residual */
  SIPG_ERR_TIMEOUT = -7,   /* a bounded wait ran out */
  SIPG_ERR_STATE = -8      /* call out of order (e.g. solve before viscosity) */
};

enum { SIPG_BC_DIRICHLET = 0, SIPG_BC_NEUMANN = 1 };
enum { SIPG_OP_VISCOUS = 0, SIPG_OP_POISSON = 1 };
/* Arithmetic of an apply: SIPG_F64 native binary64; SIPG_F32 binary32;
 * SIPG_F64_FF binary64 storage with float-float arithmetic (each value an
 * unevaluated sum of two binary32 numbers, ~48-bit significand), which runs on
 * the FP32 pipe and matches the FP64 result to ~1e-14 relative. */
enum { SIPG_F64 = 0, SIPG_F32 = 1, SIPG_F64_FF = 2 };
enum { SIPG_FACE_NU_MAX = 0, SIPG_FACE_NU_ARITH = 1, SIPG_FACE_NU_HARMONIC = 2 };
enum { SIPG_LAW_CONSTANT = 0, SIPG_LAW_ANALYTIC = 1, SIPG_LAW_SINKER = 2, SIPG_LAW_CARREAU = 3 };
enum { SIPG_PRECOND_NONE = 0, SIPG_PRECOND_JACOBI = 1, SIPG_PRECOND_MG = 2 };
/* multigrid hierarchy below the DG level (sipg_opts.mg_cph) */
enum { SIPG_MG_AUTO = -1, SIPG_MG_DG = 0, SIPG_MG_CPH = 1 };

typedef struct sipg_ctx sipg_ctx;

/* Box mesh [0,lx]x[0,ly]x[0,lz] cut into nx*ny*nz affine hexahedra (Sec. 5).
 * Boundary types per box face in the order -x,+x,-y,+y,-z,+z; the pressure
 * types apply to the Poisson operator (Dirichlet velocity walls normally go
 * with Neumann pressure walls, Sec. 3.2). */
typedef struct {
  int nx, ny, nz;
  double lx, ly, lz;
  int bc_velocity[6];
  int bc_pressure[6];
  /* HOST, optional: positions of the (nx+1)(ny+1)(nz+1) vertices of the
   * structured cells, x fastest, 3 doubles each; each cell is the trilinear
   * image of the unit cube through its 8 vertices (general hexahedra, Sec. 5;
   * the jittered channel mesh). Copied during sipg_create. NULL: the box
   * [0,lx]x[0,ly]x[0,lz] (lx, ly, lz are then ignored otherwise). On such a
   * mesh: sipg_set_viscosity, FP64 applies on every level, sipg_solve with any
   * preconditioner (the multigrid runs in FP64: mg_precision is set to
   * SIPG_F64; h-levels take every other vertex, the transfers are the
   * reference-cell embeddings); float-float and FP32 applies, mass operators,
   * the splitting step and serving return SIPG_ERR_INVALID. */
  const double* vertices;
  /* Topology beyond the plain box (zero-initialised fields keep the box):
   * active   HOST, optional: nx*ny*nz flags, x fastest, 0 = the grid cell is
   *          removed (the solid block below a backward-facing step, say); NULL =
   *          every cell. The cells of the mesh are the active cells, numbered in
   *          grid order; every vector is laid out over them.
   * bc_removed_velocity, bc_removed_pressure: condition on faces against a
   *          removed cell (velocity Dirichlet with zero wall velocity and
   *          pressure Neumann for a wall).
   * periodic[3]: 1 = direction d is periodic (each direction needs >= 2 cells;
   *          the bc of its two sides is unused); the first and last cell layers
   *          are face neighbours.
   * origin[3]: the grid's lower corner (positions of nodes, viscosity laws).
   * Removed cells or periodic directions: no cph hierarchy; with vertices the
   * active cells are trilinear (the jittered channel; the vertex array covers the
   * whole grid and the vertices of a periodic direction's end layers must agree
   * up to the period); multigrid h-levels coarsen while every 2x2x2 block of
   * cells is all active or all removed. */
  const unsigned char* active;
  int bc_removed_velocity, bc_removed_pressure;
  int periodic[3];
  double origin[3];
} sipg_mesh_desc;

/* Discretisation and solver options. Zero-initialised fields take the
 * defaults in brackets (sipg_default_opts fills them in explicitly).
 *  k_u            velocity degree, 2..5 (pressure degree k_u - 1) [3]
 *  penalty_factor C_IP of tau = C_IP (k+1)^2 max(Lambda-,Lambda+) nubar;
 *                 the paper takes tau "from Hillewaert 2013" without
 *                 printing it (Sec. 5.1, 5.2) [1.0]
 *  face_nu        nubar on a face point: SIPG_FACE_NU_* [MAX]
 *  mg_precision   arithmetic of the multigrid V-cycle, SIPG_F32 / SIPG_F64
 *                 (the paper: single precision, Sec. 5.4) [F32]
 *  cheb_degree    Chebyshev-Jacobi smoother degree [3]
 *  cheb_range     lmax / lmin of the smoother interval [20]
 *  cheb_lmax_factor  safety factor on the Lanczos estimate [1.2]
 *  lanczos_steps  Lanczos steps of the eigenvalue estimate [15]
 *  coarse_max_dofs   direct solve below this many unknowns (Sec. 5.4) [2000]
 *  seed           seed of the Lanczos start vector [0]
 *  krylov_arith   arithmetic of the outer CG's operator applies [F64] */
typedef struct {
  int k_u;
  double penalty_factor;
  int face_nu;
  int mg_precision;
  int cheb_degree;
  double cheb_range;
  double cheb_lmax_factor;
  int lanczos_steps;
  int coarse_max_dofs;
  uint64_t seed;
  int krylov_arith;  /* arithmetic of the FP64 operator applies inside CG:
                        SIPG_F64 or SIPG_F64_FF [F64] */
  int mg_cph;        /* SIPG_MG_CPH: "cph" hierarchy of Sec. 5.4 - below the DG level,
                        the continuous space of the same degree, then lower degrees and
                        coarser meshes in the continuous space (Galerkin operators
                        P^T A_DG P); plain boxes only (no vertex array, no removed
                        cells, no periodic direction: SIPG_ERR_INVALID otherwise).
                        SIPG_MG_DG: DG on every level. SIPG_MG_AUTO: cph on a plain
                        box, DG on any other mesh [AUTO from sipg_default_opts; a
                        zero-filled struct reads as DG] */
  int mg_setup_lag;  /* multigrid setup after a viscosity update: the level diagonals
                        are rebuilt at every update, the Chebyshev eigenvalue
                        estimates and the coarse-level inverse at every mg_setup_lag-th
                        update (and whenever the mass coefficient changes); between
                        full rebuilds the preconditioner keeps the earlier ones - a
                        fixed SPD preconditioner per solve, so the CG solution is
                        unchanged, only its iteration count may grow [1 = rebuild at
                        every update; 0 is read as 1] */
} sipg_opts;

/* Viscosity field (Eq. viscosity_general and Sec. 2).
 *  CONSTANT  nu
 *  ANALYTIC  nu(x) = 1 + 9 sin^2(pi x) sin^2(pi y) sin^2(pi z)
 *  SINKER    n_spheres spheres (centers: HOST array of 3*n_spheres doubles,
 *            copied during the call), radius, nu_max inside, nu_matrix
 *            outside; projected onto one constant per cell (element-local L2
 *            projection with the cell's Gauss rule)
 *  CARREAU   eta(gdot) = eta_inf + (eta0 - eta_inf) (kappa + (lambda gdot)^a)^((b-1)/a),
 *            gdot = sqrt(2 eps(u):eps(u)) of the linearization velocity */
typedef struct {
  int law;
  double nu;
  int n_spheres;
  const double* centers;
  double radius, nu_max, nu_matrix;
  double eta0, eta_inf, kappa, lambda, a, b;
} sipg_rheology;

typedef struct {
  double rtol;      /* relative residual target ||b - A x|| <= rtol ||b|| [1e-8] */
  double atol;      /* absolute residual target [0] */
  int maxit;        /* iteration limit [500] */
  int precond;      /* SIPG_PRECOND_* [MG] */
  double mass_coeff;/* m of the operator m M + A (viscous step, gamma0/dt) [0] */
} sipg_solve_opts;

typedef struct {
  int iterations;
  double rel_residual;   /* final ||r|| / ||b|| (recomputed, not recursive) */
  double seconds;        /* wall time of the solve (host clock, sync) */
  int status;            /* SIPG_OK or SIPG_ERR_* */
} sipg_solve_stats;

/* Fill *o with the defaults listed above. */
void sipg_default_opts(sipg_opts* o);

/* Create a context on the current CUDA device. Builds the multigrid level
 * hierarchies of both operators (p-levels k -> 2 -> 1 of the velocity,
 * k_p -> ... -> 1 of the pressure, then h-levels until fewer than
 * coarse_max_dofs unknowns or an odd cell count, Sec. 5.4) and allocates
 * their storage. Errors: SIPG_ERR_INVALID for k_u outside 2..5, non-positive
 * sizes or bad boundary types; SIPG_ERR_NOMEM when the device is full. */
int sipg_create(const sipg_mesh_desc* mesh, const sipg_opts* opts, void* stream, sipg_ctx** out);
int sipg_destroy(sipg_ctx* ctx);
const char* sipg_last_error(const sipg_ctx* ctx);

/* Sizes: DoFs of a level's vector (level 0 = the fine space) and the level
 * count of an operator's hierarchy. */
int sipg_num_levels(const sipg_ctx* ctx, int op, int* n_levels);
int sipg_level_info(const sipg_ctx* ctx, int op, int level, int* cells_xyz /*3*/, int* degree,
                    int64_t* n_dofs);

/* Evaluate the viscosity at the cell and face quadrature points of every
 * multigrid level (Eq. viscosity_pointwise; Sec. 5.4: nu is stored at the
 * integration points of each level and refreshed through the transfer
 * operators when the linearization changes), then rebuild the inverse
 * diagonals, the Chebyshev eigenvalue estimates and the coarse-level inverse
 * of BOTH operators. u_lin: DEVICE FP64 velocity vector of the fine level,
 * required for CARREAU, ignored otherwise. (sync) */
int sipg_set_viscosity(sipg_ctx* ctx, const sipg_rheology* rh, const double* u_lin);

/* y = (mass_coeff M + A) x on the fine level of operator op (A_visc of
 * Eq. viscous_term_weak, or the SIPG Laplacian of Eq. pressure_step_weak).
 * prec SIPG_F64 or SIPG_F64_FF: x, y DEVICE double*; SIPG_F32: DEVICE float*.
 * x and y must not overlap. */
int sipg_apply(sipg_ctx* ctx, int op, int prec, const void* x, void* y, double mass_coeff);

/* Same as sipg_apply with FP64 HOST buffers: copies x to the device, applies,
 * copies y back (sync). */
int sipg_apply_host(sipg_ctx* ctx, int op, const double* x_host, double* y_host, double mass_coeff);

/* Same as sipg_apply_host without any device allocation, for callers that
 * cannot let a library call allocate device memory (a caller whose memory
 * pool or caching allocator owns the device budget, or a host-memory-only
 * plain-C caller). No counterpart in the paper: it is an interface service.
 * x and y are staged in one fixed device array of 524,288 doubles per vector
 * (8 MiB, reserved on every GPU that loads the library until exit); a larger
 * fine level is rejected with SIPG_ERR_INVALID. All calls on a device share
 * that array, so calls that overlap on the GPU race: serialise them. The
 * first call on a device looks up the array's device address; make it before
 * any stream capture. The device that was current at sipg_create must be
 * current at the call, else SIPG_ERR_INVALID (nothing is copied). (sync) */
int sipg_apply_host_static(sipg_ctx* ctx, int op, const double* x_host, double* y_host, double mass_coeff);

/* Level-operator apply on multigrid level `level` (level 0 = fine). */
int sipg_level_apply(sipg_ctx* ctx, int op, int level, int prec, const void* x, void* y,
                     double mass_coeff);

/* Solve (mass_coeff M + A) x = b with FP64 CG (Sec. 5.4), preconditioned by
 * nothing, the FP64 Jacobi diagonal, or the hp-multigrid V-cycle whose
 * arithmetic is opts.mg_precision. b, x: DEVICE double*; x holds the initial
 * guess on entry and the solution on return. For the all-Neumann Poisson
 * operator, b and the iterates are kept mean-free (Sec. 3.2: the pressure is
 * fixed up to a constant). Convergence of the recursive residual is confirmed
 * with the true residual b - A x; when that is still above the tolerance, CG
 * restarts from it (at most three times, within maxit). stats->rel_residual is
 * the true relative residual of the returned x. (sync) */
int sipg_solve(sipg_ctx* ctx, int op, const double* b, double* x, const sipg_solve_opts* so,
               sipg_solve_stats* stats);

/* y = coeff M x with the cell mass matrix M of operator op (the element-local
 * L2 inner product (v, u)_{Omega_e} of Eqs. convective_step_weak,
 * projection_step_weak and viscous_step_weak, k+1 point Gauss rule); M is
 * block diagonal over cells. prec as for sipg_apply. x and y may be the same
 * buffer. */
int sipg_mass_apply(sipg_ctx* ctx, int op, int prec, const void* x, void* y, double coeff);

/* y = (coeff M)^-1 x: the "simple mass matrix solve" of the convective and
 * projection steps (Sec. 3.2), exact and cell-local (tensor product of the 1D
 * inverse mass matrix on the affine box). coeff != 0. x and y may alias. */
int sipg_inverse_mass_apply(sipg_ctx* ctx, int op, int prec, const void* x, void* y, double coeff);

/* ------------------------------------------- nonlinear viscous step (Alg. 1) */
typedef struct {
  double mass_coeff; /* gamma_0/dt of the viscous step operator (gamma_0/dt) M + A(nu) [0] */
  double rtol;       /* eps_nl^rel: stop when ||r^k|| <= rtol ||r^0|| [1e-6] */
  double atol;       /* eps_nl^abs: ... or when ||r^k|| <= atol [1e-12] */
  int maxit;         /* N_nl, the limit on Picard updates [20] */
  int aitken;        /* 1 Aitken relaxation of the updates, 0 plain Picard [1] */
  double omega_init; /* relaxation factor of the first update [1] */
  double lin_rtol;   /* each linear solve to lin_rtol times its initial residual ... [1e-3] */
  double lin_atol;   /* ... or to lin_atol, whichever is larger [0] */
  int lin_maxit;     /* CG iteration limit per solve (reaching it is not an error) [500] */
  int precond;       /* SIPG_PRECOND_* of the linear solves [MG] */
} sipg_picard_opts;

typedef struct {
  int iterations;     /* Picard updates made (= linear solves) */
  int lin_iterations; /* CG iterations summed over the linear solves */
  double res0;        /* ||r^visc,0|| */
  double res;         /* ||r^visc|| of the returned iterate */
  double seconds;     /* wall time (host clock, sync) */
  int status;         /* SIPG_OK converged; SIPG_ERR_MAXIT maxit updates without converging */
  int history_len;    /* capacity of the two optional arrays below (0: none) */
  double* residuals;  /* HOST, optional: ||r^k||, k = 0..iterations */
  double* omegas;     /* HOST, optional: relaxation factor of update k = 0..iterations-1 */
} sipg_picard_stats;

/* Fill *o with the defaults listed above. */
void sipg_default_picard_opts(sipg_picard_opts* o);

/* Viscous step with a velocity-dependent viscosity (Sec. 5.4, Alg. 1 with the
 * convective term explicit): find u with
 *     r(u) = b - ((gamma_0/dt) M + A(nu(u))) u = 0,  nu(u) = eta(gamma_dot(eps(u)))
 * by Picard updates of the viscosity (Eq. viscosity_pointwise) and linear
 * solves of the viscous step, the iterates relaxed by Aitken's factor
 *     omega_k = -omega_{k-1} r_{k-1}.(r_k - r_{k-1}) / ||r_k - r_{k-1}||^2
 * computed from the full nonlinear residuals r_k = r(u^k). Stops as soon as
 * ||r^k|| <= rtol ||r^0|| or ||r^k|| <= atol. Each linear solve is the CG of
 * sipg_solve started from u^k (its initial residual is r^k).
 * b, u: DEVICE double* on the fine velocity level; u holds the initial guess
 * (the extrapolation u#) on entry and the last iterate on return. On return
 * the stored viscosity is nu(u). The first call allocates four fine-level
 * work vectors that live as long as the context. (sync) */
int sipg_picard_solve(sipg_ctx* ctx, const sipg_rheology* rh, const double* b, double* u,
                      const sipg_picard_opts* po, sipg_picard_stats* stats);

/* ------------------------------------ one step of the projection scheme */
/* Box with velocity-Dirichlet walls on all six sides (pressure Neumann there),
 * steady wall velocity g constant per box side (no-slip walls: zero; a
 * lid-driven cavity: the lid's tangential velocity), convective term explicit
 * (Sec. 3.2 / 5.1, Alg. 1):
 *  1 convective step  (gamma0/dt) M uhat = M b + sum_i alpha_i/dt M u^{n-i}
 *                                          - sum_i beta_i C(u^{n-i}),
 *    C = c_h(., u; u) of Eq. (convective_term_weak) with the upwind flux;
 *  2 pressure step    SIPG Laplacian p = (gamma0/dt)[(grad q, uhat) - (q, {{uhat}}.n)],
 *    on the walls the consistent Neumann datum h_p (Eq. pressure_Neumann_BC,
 *    vorticity and viscosity by element-local L2 projection onto Q_k) against
 *    g_uhat (Eq. guhat_consistent_BC); solved by MG-CG, mean-free;
 *  3 projection step  (gamma0/dt) M uhathat = (gamma0/dt) M uhat + (div v, p) - (v, {{p}} n);
 *  4 viscous step     ((gamma0/dt) M + A(nu)) u^{n+1} = (gamma0/dt) M uhathat + wall-data terms,
 *    nu = eta(gamma_dot(eps(u#))) with u# the extrapolation of order m (linear
 *    implicit), or the Picard/Aitken loop of sipg_picard_solve (implicit; zero
 *    wall velocity only).
 * BDF1 for the first step after sipg_step_init, BDF2 afterwards (gamma0 = 3/2,
 * alpha = (2, -1/2), beta = (2, -1)). Laws: SIPG_LAW_CONSTANT or SIPG_LAW_CARREAU.
 * Walls: every boundary id present is velocity Dirichlet with pressure Neumann
 * (walls, inflow) or velocity Neumann with pressure Dirichlet (outflow, p = 0,
 * traction free); periodic directions and removed cells (the channel behind a
 * backward-facing step) are allowed. With time-dependent wall data d_t g is the
 * BDF approximation of the step, which leaves g(t_{n+1}) alone in the pressure
 * datum. */
enum { SIPG_VISC_LINEAR_IMPLICIT = 0, SIPG_VISC_IMPLICIT = 1 };
enum { SIPG_CONV_EXPLICIT = 0, SIPG_CONV_LINEAR_IMPLICIT = 1 };
enum { SIPG_FIELD_U = 0, SIPG_FIELD_P = 1, SIPG_FIELD_UHAT = 2, SIPG_FIELD_UHATHAT = 3, SIPG_FIELD_PPE_RHS = 4,
       SIPG_FIELD_U_PREV = 5 };

typedef struct {
  double dt;                 /* time step (constant; sipg_cfl_dt gives Eq. CFL_timestep_selection) */
  double wall_velocity[18];  /* g on box sides -x,+x,-y,+y,-z,+z (3 components each) [0] */
  const double* body;        /* DEVICE body force b_h on the velocity space, or NULL [NULL] */
  int viscosity_mode;        /* SIPG_VISC_* [LINEAR_IMPLICIT] */
  int convective_mode;       /* SIPG_CONV_EXPLICIT (alpha_c = 0) or SIPG_CONV_LINEAR_IMPLICIT
                                (alpha_c = 1, u* = u#: c_h(v, u^{n+1}; u#) in the viscous step,
                                solved by GMRES; linear-implicit viscosity only) [EXPLICIT] */
  int gmres_restart;         /* GMRES restart length [30] */
  double ppe_rtol;           /* pressure CG: ||r|| <= ppe_rtol ||rhs|| [1e-8] */
  double visc_rtol;          /* viscous CG (linear implicit) [1e-8] */
  int maxit;                 /* CG iteration limit of both [1000] */
  sipg_picard_opts picard;   /* SIPG_VISC_IMPLICIT: mass_coeff is set by the step */
  int penalty;               /* 1: end the step with the divergence and continuity penalty
                                step (sipg_penalty_step, factors 1) [0] */
  double penalty_rtol;       /* its CG tolerance [1e-10] */
  const double* wall_points;      /* DEVICE or NULL: wall velocity g(t_{n+1}) at the Gauss points of
                                     every boundary face, [nbf][n^2][3] (sipg_boundary_points gives
                                     the positions); replaces wall_velocity [NULL] */
  const double* wall_points_prev; /* DEVICE or NULL: g(t_n) likewise, for the convective term of
                                     u^n (NULL: wall_points, steady data) [NULL] */
} sipg_step_opts;

typedef struct {
  int order;                                  /* BDF order of this step */
  int ppe_iterations, visc_iterations;        /* CG iterations (viscous: summed over Picard updates) */
  int picard_updates;
  double ppe_rel_residual, visc_rel_residual; /* final relative residuals (Picard: ||r||/||r0||) */
  double t_convective, t_pressure, t_projection, t_viscous, seconds; /* host clock, synchronised */
  int status;
  int penalty_iterations;                     /* CG iterations of the penalty step (0 without) */
  double t_penalty;                           /* its host-clock seconds (within seconds) */
} sipg_step_stats;

void sipg_default_step_opts(sipg_step_opts* o);

/* Start a run from u0 (DEVICE velocity, fine level) and p0 (DEVICE pressure or
 * NULL for zero); the first call allocates the step's vectors (about ten
 * velocity vectors; they live as long as the context). */
int sipg_step_init(sipg_ctx* ctx, const double* u0, const double* p0);

/* Advance one time step (sync). */
int sipg_step(sipg_ctx* ctx, const sipg_rheology* rh, const sipg_step_opts* so, sipg_step_stats* stats);

/* Copy a field of the current state or of the last step to a DEVICE buffer:
 * U (u^n), U_PREV (u^{n-1}), P (p^n), UHAT, UHATHAT, PPE_RHS (the pressure
 * step's right-hand side before the mean is removed). */
int sipg_step_field(sipg_ctx* ctx, int which, double* out);

/* Boundary faces of the velocity mesh (fine level): *nbf their number; with
 * cell_face_id (HOST, 3 ints per face) their cell, face (-x,+x,-y,+y,-z,+z) and
 * boundary id (0..5 the grid's sides, 6 faces against removed cells), in the
 * order of the wall_points arrays; with xyz (DEVICE, nbf * n^2 * 3 doubles) the
 * positions of their n^2 Gauss points (point a + n b over the face's
 * tangential directions t1 < t2). Either pointer may be NULL. (sync) */
int sipg_boundary_faces(sipg_ctx* ctx, int* nbf, int* cell_face_id, double* xyz);

/* dt = courant / k_u^1.5 / max over cells and Gauss points of |J^-1 u|
 * (Eq. CFL_timestep_selection); u: DEVICE velocity. Returns SIPG_ERR_INVALID
 * (dt untouched) for a zero field. (sync) */
int sipg_cfl_dt(sipg_ctx* ctx, const double* u, double courant, double* dt);

/* The forms on their own (DEVICE vectors of the fine level):
 * y = C(u) for wall velocity wall_g (18 host doubles, NULL for no-slip);
 * y = (div v, p) - (v, {{p}} n) for a pressure p; y = wall-data terms of the
 * viscous form with the stored level-0 viscosity. */
int sipg_convective_apply(sipg_ctx* ctx, const double* wall_g, const double* u, double* y);
int sipg_projection_rhs(sipg_ctx* ctx, const double* p, double* y);
/* y = sum_e c_h(v, u; w): the convective form linear in u for a fixed transport
 * velocity w, walls u^+ = -u^- + 2 wall_u, w^+ = -w^- + 2 wall_w (18 host
 * doubles each, NULL = 0). */
int sipg_convective_lin_apply(sipg_ctx* ctx, const double* w, const double* wall_w, const double* wall_u,
                              const double* u, double* y);
int sipg_viscous_wall_rhs(sipg_ctx* ctx, const double* wall_g, double* y);

/* Solve ((mass_coeff M + A(nu)) + C(w)) x = b, C(w) u = sum_e c_h(v, u; w) the
 * upwind convective form of Eq. (convective_term_weak) linear in u for the
 * transport velocity w (DEVICE, fine velocity level; NULL: no convective
 * term): the viscous step with the linearly implicit convective term
 * (alpha_c = 1, u* = u#, Eq. viscous_step_with_convection). The operator is
 * not symmetric: restarted GMRES(restart) with right preconditioning by so->
 * precond (the multigrid V-cycle of the symmetric part mass_coeff M + A).
 * Homogeneous wall data for x; wall_w (18 host doubles or NULL) is w's wall
 * velocity. The first call allocates restart + 4 fine-level vectors. (sync) */
int sipg_solve_convective(sipg_ctx* ctx, const double* w, const double* wall_w, const double* b, double* x,
                          const sipg_solve_opts* so, int restart, sipg_solve_stats* stats);

/* ------------------------------------------------- manufactured solutions
 * Load vectors of the manufactured solutions that verify the operators (Sec. 7.1
 * checks convergence with manufactured solutions; here the steady operators):
 * b_i = integral of phi_i f over each cell, over-integrated with k+4 Gauss points
 * per direction, on the fine level of the viscous (SIPG_MMS_VELOCITY) or Poisson
 * (SIPG_MMS_PRESSURE) space; b: DEVICE vector of that space.
 *   SIPG_MMS_VELOCITY: u = s(x) (1, -1, 2), s = sin(pi x) sin(pi y) sin(pi z), with
 *     the analytic viscosity nu = 1 + 9 s^2 (SIPG_LAW_ANALYTIC): f = -div(2 nu eps(u));
 *     u = 0 on the walls of the unit cube.
 *   SIPG_MMS_PRESSURE: p = cos(pi x) cos(pi y) cos(pi z), f = -lap p = 3 pi^2 p;
 *     zero normal derivative on the walls of the unit cube, zero mean.
 * Affine cells only (SIPG_ERR_INVALID with vertices). (sync) */
enum { SIPG_MMS_VELOCITY = 0, SIPG_MMS_PRESSURE = 1 };
int sipg_rhs_manufactured(sipg_ctx* ctx, int case_id, double* b);

/* ------------------------------------ divergence and continuity penalty step
 * Sec. 3.2, Eq. (penalty_step), the last sub-step of Alg. 1: the velocity u of
 * the viscous step becomes u~, the solution of
 *   (v, u~) + (div v, tau_div,e div u~) + (v.n, tau_F (u~^- - u~^+).n) = (v, u)
 * for all v, tau_F the mean of the two cells' tau_cont,e on interior faces and
 * tau_cont,e on a Dirichlet wall, where u~^+ is the wall velocity (18 host
 * doubles, sides -x,+x,-y,+y,-z,+z, NULL = 0). The paper takes the penalty
 * parameters from Fehn et al. (2018) without printing them; this library uses
 *   tau_div,e = zeta_div ubar_e h_e / (k+1) dt,  tau_cont,e = zeta_cont ubar_e dt,
 * ubar_e the cell mean of |u|, h_e = |Omega_e|^(1/3) (zeta = 1 in sipg_step).
 * Box meshes, velocity degree 2..5; all vectors DEVICE, fine velocity level.
 *
 * sipg_penalty_tau: tau_div, tau_cont (n_cells doubles each) from u.
 * sipg_penalty_apply: y = K x, K the left-hand side above (x != y).
 * sipg_penalty_wall_rhs: y = the wall-data part of the right-hand side.
 * sipg_penalty_step: u_out = u~ by CG preconditioned with the inverse cell mass
 *   matrix, started from u, ||b - K u_out|| <= rtol ||b||; u_out may equal u.
 *   SIPG_ERR_MAXIT when maxit iterations do not reach rtol. The first call
 *   allocates five velocity vectors. (sync) */
int sipg_penalty_tau(sipg_ctx* ctx, const double* u, double dt, double zeta_div, double zeta_cont,
                     double* tau_div, double* tau_cont);
int sipg_penalty_apply(sipg_ctx* ctx, const double* tau_div, const double* tau_cont, const double* x, double* y);
int sipg_penalty_wall_rhs(sipg_ctx* ctx, const double* wall_g, const double* tau_cont, double* y);
int sipg_penalty_step(sipg_ctx* ctx, const double* wall_g, const double* u, double dt, double zeta_div,
                      double zeta_cont, double rtol, int maxit, double* u_out, int* iterations,
                      double* rel_residual);

/* ------------------------------------------------ multigrid pieces (tests) */
/* Test hook for the float-float conversions of the SIPG_F64_FF kernels' loads
 * and stores: hilo[2i], hilo[2i+1] = (RN(x_i), RN(x_i - RN(x_i))) as binary32,
 * back[i] = hi + lo rounded to binary64. DEVICE buffers of n doubles, 2n
 * floats and n doubles, on the context's stream (sync). */
int sipg_ff_convert(sipg_ctx* ctx, const double* x, float* hilo, double* back, int64_t n);

/* Host-only test hooks of the grid topology (no GPU needed): for an nx x ny x nz
 * grid with active flags (HOST, x fastest, NULL = every cell) and periodic[3],
 * sipg_topology_tables sets *ncells and *nbf and, where the pointers are not NULL,
 * fills nbr (6 * ncells ints: the cell across each face, or -1 - (boundary id +
 * 8 * boundary-face number)) and bface (nbf ints: cell * 6 + face), the tables the
 * kernels read. sipg_coarsen_mask writes the active flags of the once-coarsened
 * grid (nx/2 x ny/2 x nz/2) and returns 1, or returns 0 when a 2x2x2 block mixes
 * active and removed cells. */
int sipg_topology_tables(int nx, int ny, int nz, const unsigned char* active, const int* periodic, int* ncells,
                         int* nbf, int* nbr, int* bface);
int sipg_coarsen_mask(int nx, int ny, int nz, const unsigned char* fine, unsigned char* coarse);

/* Host-only test hook: the multigrid level sequence sipg_create would build for this
 * mesh and these options, without allocating (a dry run of the hierarchy):
 * *nlevels levels of operator op; with info (HOST, 6 ints per level, at most
 * max_levels) the grid nx, ny, nz, the degree, the active cells and the DoFs
 * (clamped to INT_MAX) of each level, finest first. */
int sipg_level_plan(const sipg_mesh_desc* mesh, const sipg_opts* opts, int op, int max_levels, int* nlevels,
                    int* info);

/* Copy the stored viscosity of a level to DEVICE buffers: nu_cell
 * [cells][n^3] and nu_face [cells][6][n^2] (the cell's own side of each face;
 * faces -x,+x,-y,+y,-z,+z; face point a + n b over the face's tangential
 * directions in increasing order). */
int sipg_get_viscosity(const sipg_ctx* ctx, int level, double* nu_cell, double* nu_face);
/* FP64 inverse diagonal of a level operator (with mass_coeff of the last
 * set_viscosity / solve call: 0 unless a solve set it) into a DEVICE buffer. */
int sipg_get_inverse_diagonal(const sipg_ctx* ctx, int op, int level, double* out);
/* Largest eigenvalue estimate of D^-1 A on a level (before the 1.2 factor). */
int sipg_get_lmax_estimate(const sipg_ctx* ctx, int op, int level, double* lmax);
/* Prolongate level+1 -> level (dir = +1) or restrict level -> level+1
 * (dir = -1, the transpose). DEVICE buffers of precision prec. */
int sipg_transfer(sipg_ctx* ctx, int op, int level, int dir, int prec, const void* in, void* out);
/* One Chebyshev-Jacobi smoother application on a level: x <- S(x, b),
 * DEVICE buffers of precision prec, x updated in place. */
int sipg_smooth(sipg_ctx* ctx, int op, int level, int prec, const void* b, void* x);
/* One V-cycle x = V(b) from a zero initial guess, FP64 DEVICE buffers on
 * level 0 (internally in opts.mg_precision). */
int sipg_vcycle(sipg_ctx* ctx, int op, const double* b, double* x);
/* Physical coordinates of the Gauss-Lobatto nodes of a level into a HOST
 * buffer [cells][n^3][3] (for building interpolated input fields). */
int sipg_node_points(const sipg_ctx* ctx, int op, int level, double* xyz_host);

/* Device bytes sipg_create would allocate for this mesh and options
 * (no allocation; used for admission by HBM budget). */
int sipg_estimate_bytes(const sipg_mesh_desc* mesh, const sipg_opts* opts, int64_t* bytes);

/* ---------------------------------------------------------- measurement
 * FMA throughput of the current device's FP64 (prec SIPG_F64) or FP32
 * (SIPG_F32) pipe in TFLOP/s (2 flops per multiply-add): independent FMA
 * chains on every SM, timed with CUDA events after a warm-up launch. It is the
 * ALU denominator of the benchmark's roofline fractions (the paper has no
 * counterpart: it measures on CPUs). Allocates a few KB and a private stream
 * for the call. (sync) */
int sipg_alu_peak(int prec, double* tflops);

/* ------------------------------------------------------------- serving
 * Continuous-batching solve server (a systems pattern around the solver; the paper's
 * solver is Sec. 5.4): requests are admitted when a slot is free and their
 * context fits the HBM budget, every active request advances one CG iteration
 * (FP64 CG with the FP64 operator by default, or the float-float operator;
 * FP32 or FP64 hp-multigrid V-cycle) per round, the fine-level operator
 * applies of all active requests of a degree run in one persistent launch, and
 * requests join and leave between rounds. Each request solves the viscous
 * system A(nu) x = b on the unit cube (n^3 cells, Dirichlet walls) with its
 * own viscosity field and right-hand side. One worker thread drives the GPU;
 * submit/poll/drain are thread-safe. */
typedef struct sipg_server sipg_server;
typedef struct {
  uint64_t hbm_budget_bytes; /* device bytes the server's contexts may hold */
  int max_slots;             /* requests served concurrently */
  int mg_precision;          /* SIPG_F32 (default for serving) or SIPG_F64 */
  int cheb_degree;           /* 0 = 3 */
  int krylov_arith;          /* operator of the CG iterations and the final residual:
                                SIPG_F64 [0, default] or SIPG_F64_FF */
} sipg_server_opts;
/* Right-hand side of a request:
 *  MANUFACTURED  b = A u* with u* uniform(-1, 1) drawn on the device from `seed`
 *                (the result also reports ||x - u*|| / ||u*||)
 *  BUOYANCY      b = M f, M the cell mass matrix, f the nodal interpolant of
 *                -e_z chi(x), chi = 1 inside any sphere of a SINKER rheology
 *                (|x - c| <= r) and 0 elsewhere (a sinking-sphere load)
 *  HOST          b given in HOST memory (n_dofs doubles), copied by submit
 *  DEVICE        b given in DEVICE memory of the server's device (n_dofs
 *                doubles), copied at admission: keep it valid and unchanged
 *                until sipg_server_poll reports the request done */
enum { SIPG_RHS_MANUFACTURED = 0, SIPG_RHS_BUOYANCY = 1, SIPG_RHS_HOST = 2, SIPG_RHS_DEVICE = 3 };
typedef struct {
  int n_cells;               /* n^3 cells on the unit cube */
  int k_u;                   /* degree 2..5 */
  const sipg_rheology* rheology; /* HOST, copied by submit (sphere centers too):
                                SIPG_LAW_CONSTANT, ANALYTIC or SINKER */
  int rhs;                   /* SIPG_RHS_* */
  const double* b;           /* HOST or DEVICE right-hand side (rhs HOST / DEVICE) */
  double rtol;               /* relative residual target ||b - A x|| <= rtol ||b||: met by the
                                recursive CG residual, then confirmed with the true one (CG
                                restarts from the true residual, at most three times, when
                                it is still above the target) */
  int maxit;
  uint64_t seed;             /* of u* (rhs MANUFACTURED) */
  int keep_solution;         /* keep x for sipg_server_poll */
} sipg_request;
typedef struct {
  int status;                /* SIPG_OK, SIPG_ERR_MAXIT, SIPG_ERR_BREAKDOWN, SIPG_ERR_NOMEM, ... */
  int iterations;
  double rel_residual;       /* true ||b - A x|| / ||b|| of the returned x (krylov_arith operator) */
  double err_vs_ustar;       /* ||x - u*|| / ||u*|| (rhs MANUFACTURED; NaN otherwise) */
  int64_t n_dofs;
  double queue_s, solve_s, latency_s;  /* submit->admit, admit->done, submit->done */
} sipg_result;
int sipg_server_create(const sipg_server_opts* opts, sipg_server** out);
int sipg_server_submit(sipg_server* srv, const sipg_request* req, uint64_t* id);
/* SIPG_PENDING while queued or running; SIPG_OK with *res (and x_host filled,
 * n_dofs doubles, if the request kept its solution and x_host != NULL). */
int sipg_server_poll(sipg_server* srv, uint64_t id, sipg_result* res, double* x_host);
/* Wait until every submitted request is done (timeout_s <= 0: no limit);
 * SIPG_ERR_TIMEOUT when the limit runs out. */
int sipg_server_drain(sipg_server* srv, double timeout_s);
const char* sipg_server_last_error(const sipg_server* srv);
int sipg_server_destroy(sipg_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* SIPG_H */
