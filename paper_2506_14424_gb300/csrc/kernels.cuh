// Declarations of the kernel launchers shared by the host-side sources.
#pragma once
#include "common.cuh"

namespace sipg {

// ---- operator apply (operator.cuh instantiations)
template <typename T>
cudaError_t launch_apply(int n, int ncomp, const LevelGeom& g, const Tab& tab, const T* x, T* y,
                         const T* nu_cell, const T* nu_face, T mass, int nbatch, cudaStream_t st);
// FP64-accurate apply with float-float arithmetic (double storage)
// (nu given as (hi, lo) float pairs, see launch_split_ff)
// register-tiled FP32 operator (n = 2..4)
bool tpc_supported(int n);
cudaError_t launch_apply_tpc(int n, int ncomp, const LevelGeom& g, const Tab& tab, const float* x, float* y,
                             const float* nu_cell, const float* nu_face, float mass, int nbatch, cudaStream_t st);
cudaError_t launch_apply_ff(int n, int ncomp, const LevelGeom& g, const Tab& tab, const float2* x, double* y,
                            const float2* nu_cell, const float2* nu_face, double mass, int nbatch, cudaStream_t st);
// x of the float-float operator as (hi, lo) pairs (integer split, bit-identical to the hardware one)
cudaError_t launch_split_ff_int(int64_t n, const double* in, float2* out, cudaStream_t st);
cudaError_t launch_split_ff(int64_t n, const double* in, float2* out, cudaStream_t st);
cudaError_t launch_ff_convert(int64_t n, const double* in, float2* hilo, double* back, cudaStream_t st);
// float-float applies of several problems of one degree in one persistent launch;
// descs: device array of ApplyDesc<double, ff> (operator.cuh), tiles: (problem, cell0)
cudaError_t launch_apply_multi_ff(int n, int ncomp, const void* descs, const int2* tiles, int ntiles,
                                  const Tab& tab, cudaStream_t st);
cudaError_t launch_apply_multi_f64(int n, int ncomp, const void* descs, const int2* tiles, int ntiles,
                                   const Tab& tab, cudaStream_t st);
int op_cells_per_cta(int n, int ncomp);

// ---- cell mass matrix and its inverse (mass.cu): y = scale (M1 (x) M1 (x) M1) x per
// component and cell, or with M1^-1; arith 0 FP64, 1 FP32, 2 float-float (FP64 storage)
cudaError_t launch_cell_mass(int n, int ncomp, int ncells, const Tab& tab, int arith, bool inverse, double scale,
                             const void* x, void* y, cudaStream_t st);

// ---- viscosity (viscosity.cu)
struct RheologyDev {
  int law;  // 0 constant, 1 analytic, 2 sinker, 3 carreau
  double nu;
  int n_spheres;
  double centers[3 * 64];
  double radius, nu_max, nu_matrix;
  double eta0, eta_inf, kappa, lambda, a, b;
};
cudaError_t launch_viscosity(int n, const LevelGeom& g, const Tab& tab, const RheologyDev& rh,
                             const double* u, double* nu_cell, double* nu_face, cudaStream_t st);
cudaError_t launch_cell_nu_transfer(const LevelGeom& fine, const LevelGeom& coarse, int kind, int nf, int nc,
                                    const double* fine_cell, double* nu_cell, double* nu_face, cudaStream_t st);

// ---- forms of the splitting step (split.cu); n = velocity degree + 1 (3..6)
struct PpeBndArgs {
  int n_hist;        // m: velocity histories entering the convective terms
  double wconv[2];   // beta_i - betabar_i
  int visc;          // viscous terms of u^dd present (m_p > 0)
  double betabar[2]; // extrapolation of order m_p
  double gn_coef;    // -(gamma0/dt)
};
cudaError_t launch_convective(int n, const LevelGeom& g, const SplitTab& tab, const WallArg& wall_g,
                              const double* u, double* y, cudaStream_t st);
// y = sum_e c_h(phi, u; w), walls u^+ = -u^- + 2 wall_u, w^+ = -w^- + 2 wall_w (NULL = 0)
cudaError_t launch_convective_lin(int n, const LevelGeom& g, const SplitTab& tab, const WallArg& wall_w,
                                  const WallArg& wall_u, const double* w, const double* u, double* y,
                                  cudaStream_t st);
int n_wall_faces(const LevelGeom& g);  // boundary faces (g.nbf with topology tables)
cudaError_t launch_ppe_boundary(int n, const LevelGeom& g, const SplitTab& tab, const WallArg& wall_g,
                                const PpeBndArgs& a, const RheologyDev& rh, const double* u0, const double* u1,
                                double* sb, cudaStream_t st);
cudaError_t launch_ppe_rhs(int n, const LevelGeom& g, const SplitTab& tab, double coef, const double* uhat,
                           const double* sb, double* r, cudaStream_t st);
cudaError_t launch_projection_rhs(int n, const LevelGeom& g, const SplitTab& tab, const double* p, double* y,
                                  cudaStream_t st);
cudaError_t launch_viscous_wall_rhs(int n, const LevelGeom& g, const SplitTab& tab, const WallArg& wall_g,
                                    const double* nu_face, double* y, cudaStream_t st);
cudaError_t launch_cfl_max(int n, const LevelGeom& g, const SplitTab& tab, const double* u,
                           unsigned long long* vmax_bits, cudaStream_t st);
cudaError_t launch_boundary_points(int n, const LevelGeom& g, const SplitTab& tab, double* xyz, cudaStream_t st);

// ---- manufactured-solution loads (manufactured.cu); which 0 velocity, 1 pressure
cudaError_t launch_manufactured_load(int n, const LevelGeom& g, int which, double* b, cudaStream_t st);

// ---- divergence and continuity penalty step (penalty.cu); n = velocity degree + 1
cudaError_t launch_penalty_tau(int n, const LevelGeom& g, const SplitTab& tab, const double* u, double zeta_div,
                               double zeta_cont, double dt, double* tdiv, double* tcon, cudaStream_t st);
cudaError_t launch_penalty_apply(int n, const LevelGeom& g, const SplitTab& tab, const double* tdiv,
                                 const double* tcon, const double* x, double* y, cudaStream_t st);
// y += wall-data terms (nothing for NULL or zero wall velocity)
cudaError_t launch_penalty_wall(int n, const LevelGeom& g, const SplitTab& tab, const WallArg& wall_g,
                                const double* tcon, double* y, cudaStream_t st);

// ---- operators on trilinear cells (mapped.cu); n = degree + 1 (2..6)
// forms of the splitting step on trilinear cells (mapped_split.cu)
cudaError_t launch_mapped_convective(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                     const WallArg& wall_g, const double* u, double* y, cudaStream_t st);
cudaError_t launch_mapped_ppe_boundary(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                       const WallArg& wall_g, const PpeBndArgs& a, const RheologyDev& rh,
                                       const double* u0, const double* u1, double* sb, cudaStream_t st);
cudaError_t launch_mapped_ppe_rhs(int n, const LevelGeom& g, const SplitTab& tab, const double* verts, double coef,
                                  const double* uhat, const double* sb, double* r, cudaStream_t st);
cudaError_t launch_mapped_projection_rhs(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                         const double* p, double* y, cudaStream_t st);
cudaError_t launch_mapped_viscous_wall_rhs(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                           const double* lam, const WallArg& wall_g, const double* nu_face,
                                           double* y, cudaStream_t st);
cudaError_t launch_mapped_cfl_max(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                  const double* u, unsigned long long* vmax_bits, cudaStream_t st);
cudaError_t launch_mapped_mass(int n, int ncomp, const LevelGeom& g, const SplitTab& tab, const double* verts,
                               double coeff, bool inverse, const double* x, double* y, cudaStream_t st);
cudaError_t launch_mapped_boundary_points(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                          double* xyz, cudaStream_t st);
// metric terms of a trilinear level: cmet [C][10][n^3], fmet [C][6][13][n^2] (mapped.cu)
inline size_t mapped_cell_metric_len(int n, int ncells) { return (size_t)ncells * 10 * n * n * n; }
inline size_t mapped_face_metric_len(int n, int ncells) { return (size_t)ncells * 6 * 13 * n * n; }
cudaError_t launch_mapped_metric(int n, const LevelGeom& g, const SplitTab& tab, const double* verts, double* cmet64,
                                 float* cmet32, double* fmet64, float* fmet32, cudaStream_t st);
cudaError_t launch_mapped_apply_f32(int n, int ncomp, const LevelGeom& g, const SplitTab& tab, const float* cmet,
                                    const float* fmet, const double* lam, const float* nu_cell, const float* nu_face,
                                    double mass, const float* x, float* y, int nbatch, cudaStream_t st);
cudaError_t launch_mapped_apply(int n, int ncomp, const LevelGeom& g, const SplitTab& tab, const double* cmet,
                                const double* fmet, const double* lam, const double* nu_cell, const double* nu_face,
                                double mass, const double* x, double* y, int nbatch, cudaStream_t st);
cudaError_t launch_mapped_diagonal(int n, int ncomp, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                   const double* lam, const double* nu_cell, const double* nu_face, double mass,
                                   double* diag, cudaStream_t st);
cudaError_t launch_gather_vertices(int nxf, int nyf, int nxc, int nyc, int nzc, int stride, const double* fine,
                                   double* coarse, cudaStream_t st);
cudaError_t launch_mapped_lambda(int n, const LevelGeom& g, const SplitTab& tab, const double* verts, double* lam,
                                 cudaStream_t st);
cudaError_t launch_mapped_viscosity(int n, const LevelGeom& g, const SplitTab& tab, const double* verts,
                                    const RheologyDev& rh, const double* u, double* nu_cell, double* nu_face,
                                    cudaStream_t st);

// ---- continuous (cph) levels (cph.cu): P (gather), P^T (scatter-sum), R (pick), R^T
template <typename T>
cudaError_t launch_cg_map(int kind, const CgGrid& cg, const T* x, T* y, int nbatch, cudaStream_t st);

// ---- multigrid and vector kernels (mg.cu)
// interior_faces = false: without the interior-face terms (the diagonal of a continuous
// level is the sum over the copies of the cell and wall terms)
cudaError_t launch_diagonal(int n, int ncomp, const LevelGeom& g, const Tab& tab, const double* nu_cell,
                            const double* nu_face, double mass, double* diag, cudaStream_t st,
                            bool interior_faces = true);
template <typename T>
cudaError_t launch_p_transfer(int nf, int nc, int ncomp, int ncells, const TransferTab& tt, int dir,
                              const T* in, T* out, cudaStream_t st);
template <typename T>
cudaError_t launch_h_transfer(int n, int ncomp, const LevelGeom& fine, const LevelGeom& coarse,
                              const TransferTab& tt, int dir, const T* in, T* out, cudaStream_t st);
cudaError_t launch_p_interp_down(int nf, int nc, int ncomp, int ncells, const TransferTab& tt,
                                 const double* in, double* out, cudaStream_t st);
cudaError_t launch_h_interp_down(int n, int ncomp, const LevelGeom& fine, const LevelGeom& coarse,
                                 const TransferTab& tt, const int* child, const double* in,
                                 double* out, cudaStream_t st);

template <typename T>
cudaError_t launch_axpby(int64_t n, T a, const T* x, T b, T* y, cudaStream_t st);  // y = a x + b y
template <typename T>
cudaError_t launch_sub(int64_t n, const T* b, const T* t, T* r, cudaStream_t st);  // r = b - t
// Chebyshev step: d = c1 d + c2 dinv (b - t); x += d (x = d when first with zero guess)
template <typename T>
cudaError_t launch_cheb(int64_t n, T c1, T c2, const T* dinv, const T* b, const T* t, T* d, T* x,
                        bool x_zero, cudaStream_t st);
template <typename S, typename D>
cudaError_t launch_cast(int64_t n, const S* in, D* out, cudaStream_t st);
template <typename T>
cudaError_t launch_fill(int64_t n, T v, T* out, cudaStream_t st);
cudaError_t launch_add_scaled_f64(int64_t n, double a, const double* x, double* y, cudaStream_t st);
cudaError_t launch_mul(int64_t n, const double* a, const double* b, double* out, cudaStream_t st);
cudaError_t launch_reciprocal(int64_t n, const double* a, double* out, cudaStream_t st);
cudaError_t launch_scale(int64_t n, double a, const double* x, double* y, cudaStream_t st);  // y = a x
cudaError_t launch_sqrt(int64_t n, double* v, cudaStream_t st);
cudaError_t launch_random(int64_t n, uint64_t seed, double* out, cudaStream_t st);
// deterministic dot product into dev_out[0] (partials: >= kDotBlocks doubles)
constexpr int kDotBlocks = 304;
cudaError_t launch_dot(int64_t n, const double* a, const double* b, double* partials, double* dev_out,
                       cudaStream_t st);
cudaError_t launch_sum(int64_t n, const double* a, double* partials, double* dev_out, cudaStream_t st);
cudaError_t launch_add_const(int64_t n, const double* dev_c, double scale, double* y, cudaStream_t st);
cudaError_t launch_check_finite(int64_t n, const double* a, int* flag, cudaStream_t st);
// dense FP64 helpers for the coarse level
// probe vectors of the coloured column assembly of the coarse operator and the
// scatter of the probed products into the dense matrix (columns contiguous)
cudaError_t launch_colour_probes(int N, int dpc, int nb, const int* colour, double* out, cudaStream_t st);
cudaError_t launch_colour_scatter(int N, int C, int dpc, int nb, const int* owner, const double* Y, double* A,
                                  cudaStream_t st);
cudaError_t launch_unit_columns(int N, int j0, int ncols, double* out, cudaStream_t st);
// blocked step: pivots k0 .. k0+b-1 (b <= 16); Pinv: b*b, R: b*N float-float scratch
cudaError_t launch_gj_block(int N, int k0, int b, const float2* A, float2* B, float2* Pinv, float2* R,
                            cudaStream_t st);
cudaError_t launch_to_ff_inplace(int64_t n, double* v, cudaStream_t st);
cudaError_t launch_from_ff_inplace(int64_t n, double* v, cudaStream_t st);
cudaError_t launch_gemv(int N, const double* M, const double* x, double* y, cudaStream_t st);
cudaError_t launch_add_rank1(int N, double c, double* M, cudaStream_t st);
cudaError_t launch_node_points(int n, const LevelGeom& g, const Tab& tab, double* xyz, cudaStream_t st);

}  // namespace sipg
