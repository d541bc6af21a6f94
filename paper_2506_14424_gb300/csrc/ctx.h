// Host-side state of a libsipg context.
#pragma once
#include "../../include/sipg.h"
#include "common.cuh"

#include <string>
#include <vector>

namespace sipg {

struct RheologyDev;

struct Level {
  LevelGeom g{};
  int k = 0, n = 0;
  int64_t ndofs = 0;
  int next_kind = 0;         // transfer to level+1: 1 = p (degree), 2 = h (mesh)
  TransferTab tt{};          // prolongation tables toward level+1
  TransferTab interp{};      // downward interpolation of the linearization velocity
  int child[kMaxN] = {0};    // h: child of each coarse node (ties to child 0)
  double *nu_cell64 = nullptr, *nu_face64 = nullptr;
  float *nu_cell32 = nullptr, *nu_face32 = nullptr;
  float2 *nu_cellff = nullptr, *nu_faceff = nullptr;  // (hi, lo) split for float-float
  float2* xff = nullptr;     // level 0: x of the float-float apply split into (hi, lo) pairs
  double* ulin = nullptr;    // linearization velocity on this level (l > 0)
  double* diag64 = nullptr;
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  double lmax = 0.0;         // Lanczos estimate of lambda_max(D^-1 A)
  void* w[2][4] = {{nullptr}};  // [prec F64/F32][b, x, t, d]
  int N = 0;                 // coarsest level: dense size
  double* Ainv = nullptr;    // coarsest level: FP64 inverse (row-major)
  double* Atmp = nullptr;
  double* gjw = nullptr;     // coarsest level: blocked Gauss-Jordan scratch (16 x 16 + 16 x N pairs)
  double* verts = nullptr;   // trilinear cells: this level's vertices (device)
  bool own_verts = false;    //   allocated for this level (h-levels); p-levels share the finer one's
  double* lam = nullptr;     // trilinear cells: Lambda_e per cell with this level's Gauss rule
  double* cmet64 = nullptr;  // trilinear cells: metric terms of the cell points [C][10][n^3]
  float* cmet32 = nullptr;   //   (J^-1, w det J) and of the face points [C][6][13][n^2]
  double* fmet64 = nullptr;  //   (J^-1, unit normal, surface weight), FP64 and FP32
  float* fmet32 = nullptr;
  // continuous (cph) levels: values on the global node grid; the operator is
  // P^T A_DG P with the DG data (viscosity) of the twin level of the same mesh/degree
  bool cg = false;
  bool alias = false;        // shallow copy of a DG level (owns nothing)
  int twin = -1;
  CgGrid cgg{};
  int64_t ndg = 0;           // DoFs of the twin DG level
  void* tdg[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [prec][2] DG-sized temporaries
};

struct Hier {
  int op = 0, ncomp = 0;
  bool cph = false;          // L = [DG level 0, continuous twins of T[0..]]; T: the DG sequence
  std::vector<Level> T;
  bool singular = false;
  bool ready = false;
  double setup_mass = 0.0;
  // lagged setup (opts.mg_setup_lag): viscosity updates since the last full setup
  // (eigenvalue estimates and coarse inverse), and the mass coefficient it used
  int updates_since_full = 0;
  bool have_full = false;
  double full_mass = 0.0;
  std::vector<Level> L;
  double* cg[5] = {nullptr};  // r, z, p, q, tmp (level 0, FP64)
};

}  // namespace sipg

struct sipg_ctx {
  sipg_mesh_desc mesh{};
  std::vector<unsigned char> mask;  // active flags of the fine grid (empty: every cell)
  bool topo = false;                // removed cells or periodic directions: topology tables
  std::vector<int*> topo_dev;       // device topology tables (one allocation per mesh)
  struct TopoEntry {
    int nx, ny, nz, ncells, nbf, used;
    int* dev;
  };
  std::vector<TopoEntry> topo_cache;
  int used_ids = 0x3f;              // boundary ids present on the fine level (bit i: id i)
  sipg_opts opts{};
  cudaStream_t st = nullptr;
  sipg::Tab tabs[sipg::kMaxN + 1]{};
  sipg::Hier hier[2];
  bool have_nu = false;
  std::string err;
  double* partials = nullptr;
  double* dscal = nullptr;
  int* dflag = nullptr;
  double* hscal = nullptr;  // pinned
  double* host_x = nullptr;
  double* host_y = nullptr;
  int64_t host_n = 0;
  double* pic[4] = {nullptr};  // Picard work vectors: r_k, r_{k-1}, u^k, r_k - r_{k-1}
  sipg::SplitTab stabs[sipg::kMaxN + 1]{};
  struct GmresWork {  // GMRES Krylov basis and scratch (allocated on first use)
    std::vector<double*> V;
    double *z = nullptr, *tmp = nullptr, *r = nullptr;
    int m = 0;
    int64_t n = 0;
  } gm;
  // state of the splitting step (allocated by sipg_step_init)
  struct StepState {
    double* u[2] = {nullptr, nullptr};     // u^n, u^{n-1}
    double* conv[2] = {nullptr, nullptr};  // C(u^n), C(u^{n-1})
    double *uhat = nullptr, *uhh = nullptr, *tmp = nullptr, *usharp = nullptr, *bv = nullptr;
    double *p = nullptr, *prhs = nullptr, *sb = nullptr;
    unsigned long long* vmax = nullptr;
    int n_hist = 0;       // velocity histories held (1 after init, 2 after a step)
    bool conv1 = false;   // conv[1] holds C(u^{n-1})
    int64_t steps = 0;
  } ss;
  // divergence and continuity penalty step: tau per cell, right-hand side, CG vectors
  struct PenaltyWork {
    double *tdiv = nullptr, *tcon = nullptr, *b = nullptr, *r = nullptr, *z = nullptr, *p = nullptr,
           *q = nullptr;
    int64_t n = 0;
  } pw;
  bool mapped = false;          // trilinear cells from a vertex array (fine level only)
  double* dverts = nullptr;     // device copy of the vertices
  bool dry = false;     // size accounting only (sipg_estimate_bytes)
  int device = -1;      // CUDA device current at sipg_create (the context's device)
  int64_t bytes = 0;    // device bytes allocated by the hierarchy

  ~sipg_ctx();
  int fail(int code, const char* what, cudaError_t e = cudaSuccess);
  template <typename T>
  T* alloc(int64_t n, cudaError_t* e);
  int build_hierarchy(int op);
  int setup_level_smoother(int op, int l, double mass, bool estimate = true);
  int setup_coarse(int op, double mass);
  int coarse_colouring(const sipg::LevelGeom& g, std::vector<int>* colour, std::vector<int>* owner, int* ncolours);
  int setup_operator(int op, double mass);
  int ensure_setup(int op);
  template <typename T>
  int level_apply(int op, int l, const T* x, T* y, double mass);
  int level_apply_ff(int op, int l, const double* x, double* y, double mass);
  int krylov_apply(int op, const double* x, double* y, double mass);
  int dot(int64_t n, const double* a, const double* b, double* out_host);
  int project_mean(int64_t n, double* v);
  void sqrt_inplace(int64_t n, double* v);
  template <typename T>
  int smooth(int op, int l, bool x_zero, double mass);
  template <typename T>
  int transfer(int op, int l, int dir, const T* in, T* out);
  template <typename T>
  int vcycle(int op, int l, double mass);
  int coarse_solve64(int op);
  int precondition(int op, int kind, const double* r, double* z, double mass);
  int solve(int op, const double* b, double* x, const sipg_solve_opts* so, sipg_solve_stats* stats);
  int parse_rheology(const sipg_rheology* rh, const double* u_lin, sipg::RheologyDev* out);
  int eval_viscosity(const sipg::RheologyDev& r, const double* u_lin);
  int mass_apply(int op, int prec, const void* x, void* y, double coeff, bool inverse);
  int convective_apply_total(const double* w, const sipg::WallArg& wall_w, const double* x, double* y, double mass);
  int penalty_work();
  int penalty_solve(const sipg::WallArg& wall_g, const double* u, double dt, double zeta_div, double zeta_cont,
                    double rtol, int maxit, double* x, int* iterations, double* rel_residual);
  int gmres_solve(const double* w, const sipg::WallArg& wall_w, const double* b, double* x, const sipg_solve_opts& so,
                  int restart, sipg_solve_stats* stats);
};
