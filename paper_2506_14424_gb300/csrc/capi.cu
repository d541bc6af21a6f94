// libsipg C ABI: context, level hierarchy, viscosity update, operator apply,
// FP64 CG with a Chebyshev-smoothed hp-multigrid V-cycle (Sec. 5.4 of the
// paper: CG for the pressure and viscous steps; multigrid that lowers the
// degree, then coarsens the mesh; Chebyshev-accelerated Jacobi smoothing with
// precomputed inverse diagonals; single-precision preconditioner with a
// double-precision direct solve below 2000 unknowns).
#include "../../include/sipg.h"
#include "ctx.h"
#include "kernels.cuh"
#include "tables.h"

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>

using namespace sipg;

#define CK(expr)                                                              \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess) return ctx->fail(SIPG_ERR_CUDA, #expr, e_);        \
  } while (0)

int sipg_ctx::fail(int code, const char* what, cudaError_t e) {
  char buf[512];
  if (e != cudaSuccess)
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  else
    snprintf(buf, sizeof buf, "%s", what);
  err = buf;
  return code;
}

namespace {

// Allocate and zero on the context's stream (a plain cudaMemset runs on the
// legacy default stream, which is not ordered with non-blocking streams).
template <typename T>
T* dalloc(int64_t n, cudaError_t* e, cudaStream_t st) {
  void* p = nullptr;
  *e = cudaMalloc(&p, sizeof(T) * (size_t)std::max<int64_t>(n, 1));
  if (*e == cudaSuccess) *e = cudaMemsetAsync(p, 0, sizeof(T) * (size_t)std::max<int64_t>(n, 1), st);
  return (T*)p;
}

bool valid_bc(const int* bc) {
  for (int i = 0; i < 6; ++i)
    if (bc[i] != SIPG_BC_DIRICHLET && bc[i] != SIPG_BC_NEUMANN) return false;
  return true;
}

// Topology tables of an nx x ny x nz grid with active flags act (NULL: every
// cell) and periodic directions (see LevelGeom): boundary faces are numbered in
// cell order, faces -x,+x,-y,+y,-z,+z within a cell. used_ids: bit i set when
// some boundary face carries boundary id i.
struct HostTopo {
  int ncells = 0, nbf = 0, used_ids = 0;
  std::vector<int> nbr, cgrid, gcell, bface;
};

HostTopo host_topology(int nx, int ny, int nz, const unsigned char* act, const int* periodic) {
  HostTopo t;
  const int G = nx * ny * nz;
  t.gcell.assign(G, -1);
  for (int i = 0; i < G; ++i)
    if (!act || act[i]) {
      t.gcell[i] = (int)t.cgrid.size();
      t.cgrid.push_back(i);
    }
  t.ncells = (int)t.cgrid.size();
  t.nbr.assign((size_t)t.ncells * 6, 0);
  const int dims[3] = {nx, ny, nz};
  for (int e = 0; e < t.ncells; ++e) {
    const int gi = t.cgrid[e];
    const int ijk[3] = {gi % nx, (gi / nx) % ny, gi / (nx * ny)};
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1, s = f & 1;
      int q[3] = {ijk[0], ijk[1], ijk[2]};
      q[d] += s ? 1 : -1;
      int bid = -1;
      if (q[d] < 0 || q[d] >= dims[d]) {
        if (periodic[d])
          q[d] = (q[d] + dims[d]) % dims[d];
        else
          bid = f;
      }
      if (bid < 0) {
        const int nb = t.gcell[(q[2] * ny + q[1]) * nx + q[0]];
        if (nb >= 0) {
          t.nbr[(size_t)e * 6 + f] = nb;
          continue;
        }
        bid = 6;
      }
      t.nbr[(size_t)e * 6 + f] = -1 - (bid + 8 * t.nbf);
      t.bface.push_back(e * 6 + f);
      t.used_ids |= 1 << bid;
      ++t.nbf;
    }
  }
  return t;
}

bool mesh_topology(const sipg_mesh_desc* m) {
  return m->active != nullptr || m->periodic[0] || m->periodic[1] || m->periodic[2];
}

// SIPG_MG_AUTO: the continuous (cph) levels on a plain box, the DG levels on any other mesh
int resolved_mg_cph(int mg_cph, const sipg_mesh_desc* m) {
  if (mg_cph != SIPG_MG_AUTO) return mg_cph;
  return (m->vertices || mesh_topology(m)) ? SIPG_MG_DG : SIPG_MG_CPH;
}

// Active flags of the once-coarsened grid; false if a 2x2x2 block mixes active
// and removed cells (the mesh cannot be coarsened).
bool coarsen_mask(int nx, int ny, int nz, const std::vector<unsigned char>& fine, std::vector<unsigned char>* coarse) {
  const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
  coarse->assign((size_t)cx * cy * cz, 0);
  for (int k = 0; k < cz; ++k)
    for (int j = 0; j < cy; ++j)
      for (int i = 0; i < cx; ++i) {
        int cnt = 0;
        for (int ch = 0; ch < 8; ++ch)
          cnt += fine[((size_t)(2 * k + (ch >> 2)) * ny + 2 * j + ((ch >> 1) & 1)) * nx + 2 * i + (ch & 1)] != 0;
        if (cnt != 0 && cnt != 8) return false;
        (*coarse)[((size_t)k * cy + j) * cx + i] = cnt == 8;
      }
  return true;
}

}  // namespace

// ------------------------------------------------------------ construction
template <typename T>
T* sipg_ctx::alloc(int64_t n, cudaError_t* e) {
  const size_t bytes_n = sizeof(T) * (size_t)std::max<int64_t>(n, 1);
  bytes += (int64_t)bytes_n;
  if (dry) {
    *e = cudaSuccess;
    return nullptr;
  }
  return dalloc<T>(n, e, st);
}

int sipg_ctx::build_hierarchy(int op) {
  Hier& H = hier[op];
  H.op = op;
  H.ncomp = op == SIPG_OP_VISCOUS ? 3 : 1;
  const int k0 = op == SIPG_OP_VISCOUS ? opts.k_u : opts.k_u - 1;
  const int* bc = op == SIPG_OP_VISCOUS ? mesh.bc_velocity : mesh.bc_pressure;
  std::vector<int> ks{k0};
  if (k0 > 2) ks.push_back(2);
  if (k0 > 1) ks.push_back(1);
  const int bc_removed = op == SIPG_OP_VISCOUS ? mesh.bc_removed_velocity : mesh.bc_removed_pressure;
  int nx = mesh.nx, ny = mesh.ny, nz = mesh.nz;
  std::vector<unsigned char> lmask = mask;  // active flags of the current grid (topology meshes)
  if (topo && lmask.empty()) lmask.assign((size_t)nx * ny * nz, 1);
  int used_ids = 0x3f;                      // boundary ids on the fine level (plain box: the 6 sides)
  cudaError_t e = cudaSuccess;
  // topology tables of the current grid, shared by its levels and by both hierarchies
  using Cached = TopoEntry;
  auto fill = [&](const Cached& c, LevelGeom& g) {
    g.ncells = c.ncells;
    g.nbf = c.nbf;
    if (c.dev) {
      g.nbr = c.dev;
      g.cgrid = c.dev + (size_t)6 * c.ncells;
      g.gcell = g.cgrid + c.ncells;
      g.bface = g.gcell + (size_t)g.nx * g.ny * g.nz;
    }
    if (g.nx == mesh.nx && g.ny == mesh.ny && g.nz == mesh.nz) used_ids = c.used;
  };
  auto topology = [&](LevelGeom& g) -> int {
    for (const Cached& c : topo_cache)
      if (c.nx == g.nx && c.ny == g.ny && c.nz == g.nz) {
        fill(c, g);
        return SIPG_OK;
      }
    const HostTopo t = host_topology(g.nx, g.ny, g.nz, lmask.data(), mesh.periodic);
    if (t.ncells == 0) return fail(SIPG_ERR_INVALID, "no active cell");
    const size_t cnt = t.nbr.size() + t.cgrid.size() + t.gcell.size() + t.bface.size();
    int* dev = alloc<int>((int64_t)cnt, &e);
    if (e) return fail(SIPG_ERR_NOMEM, "alloc topology", e);
    if (dev) {
      std::vector<int> all;
      all.reserve(cnt);
      for (const std::vector<int>* v : {&t.nbr, &t.cgrid, &t.gcell, &t.bface}) all.insert(all.end(), v->begin(), v->end());
      e = cudaMemcpy(dev, all.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice);
      if (e) return fail(SIPG_ERR_CUDA, "upload topology", e);
      topo_dev.push_back(dev);
    }
    topo_cache.push_back(Cached{g.nx, g.ny, g.nz, t.ncells, t.nbf, t.used_ids, dev});
    fill(topo_cache.back(), g);
    return SIPG_OK;
  };
  int rc_level = SIPG_OK;
  auto make_level = [&](int k, int lnx, int lny, int lnz) {
    Level L{};
    L.k = k;
    L.n = k + 1;
    L.g.nx = lnx;
    L.g.ny = lny;
    L.g.nz = lnz;
    L.g.ncells = lnx * lny * lnz;
    L.g.h[0] = mesh.lx / lnx;
    L.g.h[1] = mesh.ly / lny;
    L.g.h[2] = mesh.lz / lnz;
    for (int d = 0; d < 3; ++d) L.g.ih[d] = 1.0 / L.g.h[d];
    for (int d = 0; d < 3; ++d) L.g.x0[d] = mesh.origin[d];
    for (int i = 0; i < 6; ++i) L.g.bc[i] = bc[i];
    L.g.bc[6] = bc_removed;
    L.g.cip = opts.penalty_factor;
    L.g.face_nu = opts.face_nu;
    if (topo && rc_level == SIPG_OK) rc_level = topology(L.g);
    L.ndofs = (int64_t)L.g.ncells * H.ncomp * L.n * L.n * L.n;
    return L;
  };
  H.L.clear();
  for (int k : ks) H.L.push_back(make_level(k, nx, ny, nz));
  while (H.L.back().ndofs >= opts.coarse_max_dofs && nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0) {
    if (topo) {
      bool ok = true;
      const int cd[3] = {nx / 2, ny / 2, nz / 2};
      for (int d = 0; d < 3; ++d) ok = ok && (!mesh.periodic[d] || cd[d] >= 2);
      std::vector<unsigned char> cm;
      if (!ok || !coarsen_mask(nx, ny, nz, lmask, &cm)) break;
      lmask.swap(cm);
    }
    nx /= 2;
    ny /= 2;
    nz /= 2;
    H.L.push_back(make_level(H.L.back().k, nx, ny, nz));
  }
  if (rc_level != SIPG_OK) return rc_level;
  for (size_t l = 0; l + 1 < H.L.size(); ++l) {
    Level& F = H.L[l];
    Level& C = H.L[l + 1];
    if (C.g.ncells == F.g.ncells) {
      F.next_kind = 1;
      F.tt = make_p_transfer(F.n, C.n);
      F.interp = make_p_interp_down(F.n, C.n);
    } else {
      F.next_kind = 2;
      F.tt = make_h_transfer(F.n);
      F.interp = make_h_interp_down(F.n, F.child);
    }
  }
  this->used_ids = used_ids;
  H.singular = true;  // all-Neumann operator: constants (Poisson) / rigid modes (viscous)
  for (int i = 0; i < 7; ++i)
    if ((used_ids >> i & 1) && H.L[0].g.bc[i] == SIPG_BC_DIRICHLET) H.singular = false;
  // storage
  for (size_t l = 0; l < H.L.size(); ++l) {
    Level& L = H.L[l];
    const int64_t C = L.g.ncells, n3 = (int64_t)L.n * L.n * L.n, n2 = (int64_t)L.n * L.n;
    if (op == SIPG_OP_VISCOUS) {
      L.nu_cell64 = alloc<double>(C * n3, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc nu", e);
      L.nu_face64 = alloc<double>(C * 6 * n2, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc nu", e);
      L.nu_cell32 = alloc<float>(C * n3, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc nu", e);
      L.nu_face32 = alloc<float>(C * 6 * n2, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc nu", e);
      if (l == 0) {
        L.nu_cellff = alloc<float2>(C * n3, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc nu", e);
        L.nu_faceff = alloc<float2>(C * 6 * n2, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc nu", e);
      }
      if (l > 0) { L.ulin = alloc<double>(L.ndofs, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc ulin", e); }
    }
    if (l == 0 && !mapped) {
      L.xff = alloc<float2>(L.ndofs, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc split x", e);
    }
    L.diag64 = alloc<double>(L.ndofs, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc diag", e);
    L.dinv64 = alloc<double>(L.ndofs, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc diag", e);
    L.dinv32 = alloc<float>(L.ndofs, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc diag", e);
    for (int p = 0; p < 2; ++p) {
      const size_t es = p == 0 ? sizeof(double) : sizeof(float);
      for (int v = 0; v < 4; ++v) {
        void* ptr = nullptr;
        bytes += (int64_t)(es * (size_t)L.ndofs);
        if (!dry) {
          e = cudaMalloc(&ptr, es * (size_t)L.ndofs);
          if (e == cudaSuccess) e = cudaMemsetAsync(ptr, 0, es * (size_t)L.ndofs, st);
          if (e) return fail(SIPG_ERR_NOMEM, "alloc mg work", e);
        }
        L.w[p][v] = ptr;
      }
    }
  }
  H.cph = false;
  H.T.clear();
  if (opts.mg_cph && !mapped) {
    // cph: [DG level 0, continuous twins of every DG level]; the DG levels below 0 keep
    // their viscosity storage (and ulin) for the twins
    H.cph = true;
    H.T = H.L;
    std::vector<Level> lv;
    Level d0 = H.T[0];
    d0.alias = true;
    d0.next_kind = 3;  // DG -> continuous, same mesh and degree
    lv.push_back(d0);
    for (size_t j = 0; j < H.T.size(); ++j) {
      const Level& Tj = H.T[j];
      Level c{};
      c.g = Tj.g;
      c.k = Tj.k;
      c.n = Tj.n;
      c.cg = true;
      c.twin = (int)j;
      c.cgg = CgGrid{Tj.g.nx, Tj.g.ny, Tj.g.nz, Tj.k, Tj.g.nx * Tj.k + 1, Tj.g.ny * Tj.k + 1, Tj.g.nz * Tj.k + 1,
                     H.ncomp};
      c.ndofs = (int64_t)H.ncomp * c.cgg.Gx * c.cgg.Gy * c.cgg.Gz;
      c.ndg = Tj.ndofs;
      c.nu_cell64 = Tj.nu_cell64;
      c.nu_face64 = Tj.nu_face64;
      c.nu_cell32 = Tj.nu_cell32;
      c.nu_face32 = Tj.nu_face32;
      c.next_kind = Tj.next_kind;
      c.tt = Tj.tt;
      c.diag64 = alloc<double>(c.ndofs, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc diag", e);
      c.dinv64 = alloc<double>(c.ndofs, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc diag", e);
      c.dinv32 = alloc<float>(c.ndofs, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc diag", e);
      for (int v = 0; v < 4; ++v) {
        c.w[0][v] = alloc<double>(c.ndofs, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc mg work", e);
        c.w[1][v] = alloc<float>(c.ndofs, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc mg work", e);
      }
      for (int v = 0; v < 2; ++v) {
        c.tdg[0][v] = alloc<double>(c.ndg, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc cph work", e);
        c.tdg[1][v] = alloc<float>(c.ndg, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc cph work", e);
      }
      lv.push_back(c);
    }
    H.L = lv;
  }
  {
    Level& Cl = H.L.back();
    Cl.N = (int)Cl.ndofs;
    if (Cl.ndofs > 20000) return fail(SIPG_ERR_INVALID, "coarse level too large for the dense direct solve");
    Cl.Ainv = alloc<double>((int64_t)Cl.N * Cl.N, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc coarse", e);
    Cl.Atmp = alloc<double>((int64_t)Cl.N * Cl.N, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc coarse", e);
    Cl.gjw = alloc<double>(256 + 16 * (int64_t)Cl.N, &e); if (e) return fail(SIPG_ERR_NOMEM, "alloc coarse", e);
  }
  // trilinear cells: vertices of every level (p-levels share the finer level's, h-levels
  // take every other vertex), the penalty factors with each level's Gauss rule and the
  // metric terms of the operator kernels (counted in the estimate)
  if (mapped)
    for (const Level& L : H.L)
      bytes += (int64_t)(12 * (mapped_cell_metric_len(L.n, L.g.ncells) + mapped_face_metric_len(L.n, L.g.ncells)));
  if (mapped && !dry) {
    for (size_t l = 0; l < H.L.size(); ++l) {
      Level& L = H.L[l];
      if (l == 0) {
        L.verts = dverts;
      } else if (H.L[l - 1].g.ncells == L.g.ncells) {
        L.verts = H.L[l - 1].verts;
      } else {
        const Level& F = H.L[l - 1];
        e = cudaMalloc(&L.verts, sizeof(double) * 3 * (size_t)(L.g.nx + 1) * (L.g.ny + 1) * (L.g.nz + 1));
        if (!e) e = launch_gather_vertices(F.g.nx, F.g.ny, L.g.nx, L.g.ny, L.g.nz, 2, F.verts, L.verts, st);
        if (e) return fail(SIPG_ERR_NOMEM, "level vertices", e);
        L.own_verts = true;
      }
      e = cudaMalloc(&L.lam, sizeof(double) * (size_t)L.g.ncells);
      if (!e) e = launch_mapped_lambda(L.n, L.g, stabs[L.n], L.verts, L.lam, st);
      if (e) return fail(SIPG_ERR_NOMEM, "level penalty factors", e);
      const size_t lc = mapped_cell_metric_len(L.n, L.g.ncells), lf = mapped_face_metric_len(L.n, L.g.ncells);
      e = cudaMalloc(&L.cmet64, sizeof(double) * lc);
      if (!e) e = cudaMalloc(&L.cmet32, sizeof(float) * lc);
      if (!e) e = cudaMalloc(&L.fmet64, sizeof(double) * lf);
      if (!e) e = cudaMalloc(&L.fmet32, sizeof(float) * lf);
      if (!e) e = launch_mapped_metric(L.n, L.g, stabs[L.n], L.verts, L.cmet64, L.cmet32, L.fmet64, L.fmet32, st);
      if (e) return fail(SIPG_ERR_NOMEM, "level metric terms", e);
    }
  }
  // CG vectors on level 0
  for (int v = 0; v < 5; ++v) {
    H.cg[v] = alloc<double>(H.L[0].ndofs, &e);
    if (e) return fail(SIPG_ERR_NOMEM, "alloc cg", e);
  }
  return SIPG_OK;
}

sipg_ctx::~sipg_ctx() {
  if (dry) return;
  for (Hier& H : hier) {
    if (H.cph) {
      // continuous levels own their work storage; level 0 is a copy of the DG level T[0]
      for (Level& L : H.L) {
        if (!L.cg) continue;
        cudaFree(L.diag64); cudaFree(L.dinv64); cudaFree(L.dinv32); cudaFree(L.gjw);
        for (int p = 0; p < 2; ++p) for (int v = 0; v < 4; ++v) cudaFree(L.w[p][v]);
        for (int p = 0; p < 2; ++p) for (int v = 0; v < 2; ++v) cudaFree(L.tdg[p][v]);
        cudaFree(L.Ainv); cudaFree(L.Atmp);
      }
    }
    for (Level& L : (H.cph ? H.T : H.L)) {
      cudaFree(L.nu_cell64); cudaFree(L.nu_face64); cudaFree(L.nu_cell32); cudaFree(L.nu_face32);
      cudaFree(L.nu_cellff); cudaFree(L.nu_faceff); cudaFree(L.xff);
      cudaFree(L.ulin); cudaFree(L.diag64); cudaFree(L.dinv64); cudaFree(L.dinv32); cudaFree(L.gjw);
      cudaFree(L.lam);
      cudaFree(L.cmet64); cudaFree(L.cmet32); cudaFree(L.fmet64); cudaFree(L.fmet32);
      if (L.own_verts) cudaFree(L.verts);
      for (int p = 0; p < 2; ++p) for (int v = 0; v < 4; ++v) cudaFree(L.w[p][v]);
      cudaFree(L.Ainv); cudaFree(L.Atmp);
    }
    for (double*& p : H.cg) cudaFree(p);
  }
  cudaFree(partials); cudaFree(dscal); cudaFree(dflag); cudaFree(host_x); cudaFree(host_y);
  for (double* p : pic) cudaFree(p);
  for (double* p : {ss.u[0], ss.u[1], ss.conv[0], ss.conv[1], ss.uhat, ss.uhh, ss.tmp, ss.usharp, ss.bv, ss.p,
                    ss.prhs, ss.sb})
    cudaFree(p);
  cudaFree(ss.vmax);
  for (double* p : gm.V) cudaFree(p);
  cudaFree(gm.z); cudaFree(gm.tmp); cudaFree(gm.r);
  for (double* p : {pw.tdiv, pw.tcon, pw.b, pw.r, pw.z, pw.p, pw.q}) cudaFree(p);
  for (int* p : topo_dev) cudaFree(p);
  cudaFree(dverts);
  if (hscal) cudaFreeHost(hscal);
}

extern "C" void sipg_default_opts(sipg_opts* o) {
  std::memset(o, 0, sizeof *o);
  o->k_u = 3;
  o->penalty_factor = 1.0;
  o->face_nu = SIPG_FACE_NU_MAX;
  o->mg_precision = SIPG_F32;
  o->cheb_degree = 3;
  o->cheb_range = 20.0;
  o->cheb_lmax_factor = 1.2;
  o->lanczos_steps = 15;
  o->coarse_max_dofs = 2000;
  o->seed = 0;
  o->mg_cph = SIPG_MG_AUTO;
}

extern "C" int sipg_create(const sipg_mesh_desc* mesh, const sipg_opts* opts_in, void* stream, sipg_ctx** out) {
  if (!out || !mesh) return SIPG_ERR_INVALID;
  *out = nullptr;
  sipg_opts o;
  sipg_default_opts(&o);
  if (opts_in) {
    o = *opts_in;
    sipg_opts d;
    sipg_default_opts(&d);
    if (o.penalty_factor == 0) o.penalty_factor = d.penalty_factor;
    if (o.cheb_degree == 0) o.cheb_degree = d.cheb_degree;
    if (o.cheb_range == 0) o.cheb_range = d.cheb_range;
    if (o.cheb_lmax_factor == 0) o.cheb_lmax_factor = d.cheb_lmax_factor;
    if (o.lanczos_steps == 0) o.lanczos_steps = d.lanczos_steps;
    if (o.coarse_max_dofs == 0) o.coarse_max_dofs = d.coarse_max_dofs;
    if (o.k_u == 0) o.k_u = d.k_u;
  }
  if (o.k_u < 2 || o.k_u > 5) return SIPG_ERR_INVALID;
  if (mesh->nx <= 0 || mesh->ny <= 0 || mesh->nz <= 0 || !(mesh->lx > 0) || !(mesh->ly > 0) || !(mesh->lz > 0))
    return SIPG_ERR_INVALID;
  if ((int64_t)mesh->nx * mesh->ny * mesh->nz > (int64_t)1 << 28) return SIPG_ERR_INVALID;
  if (!valid_bc(mesh->bc_velocity) || !valid_bc(mesh->bc_pressure)) return SIPG_ERR_INVALID;
  if (o.mg_precision != SIPG_F32 && o.mg_precision != SIPG_F64) return SIPG_ERR_INVALID;
  if (o.face_nu < 0 || o.face_nu > 2 || o.cheb_degree < 1 || o.lanczos_steps < 2) return SIPG_ERR_INVALID;
  if (o.krylov_arith != SIPG_F64 && o.krylov_arith != SIPG_F64_FF) return SIPG_ERR_INVALID;
  if (mesh->vertices && o.krylov_arith != SIPG_F64) return SIPG_ERR_INVALID;  // FP64 applies only
  if (o.mg_cph != SIPG_MG_AUTO && o.mg_cph != SIPG_MG_DG && o.mg_cph != SIPG_MG_CPH) return SIPG_ERR_INVALID;
  if (o.mg_setup_lag < 0) return SIPG_ERR_INVALID;
  const bool topo = mesh_topology(mesh);
  o.mg_cph = resolved_mg_cph(o.mg_cph, mesh);
  if (o.mg_cph && mesh->vertices) return SIPG_ERR_INVALID;  // continuous levels: box meshes only
  if (topo) {
    if (o.mg_cph) return SIPG_ERR_INVALID;  // continuous levels: plain boxes only
    const int dims[3] = {mesh->nx, mesh->ny, mesh->nz};
    for (int d = 0; d < 3; ++d)
      if ((mesh->periodic[d] != 0 && mesh->periodic[d] != 1) || (mesh->periodic[d] && dims[d] < 2))
        return SIPG_ERR_INVALID;
    for (int b : {mesh->bc_removed_velocity, mesh->bc_removed_pressure})
      if (b != SIPG_BC_DIRICHLET && b != SIPG_BC_NEUMANN) return SIPG_ERR_INVALID;
  }
  sipg_ctx* ctx = new sipg_ctx();
  ctx->mesh = *mesh;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) ctx->device = -1;
  ctx->topo = topo;
  if (mesh->active) ctx->mask.assign(mesh->active, mesh->active + (size_t)mesh->nx * mesh->ny * mesh->nz);
  ctx->mesh.active = nullptr;  // copied above
  ctx->mesh.vertices = nullptr;  // the caller's array is copied below, not kept
  ctx->mapped = mesh->vertices != nullptr;
  ctx->opts = o;
  ctx->st = (cudaStream_t)stream;
  for (int n = 2; n <= kMaxN; ++n) ctx->tabs[n] = make_tab(n);
  for (int n = 2; n <= kMaxN; ++n) ctx->stabs[n] = make_split_tab(n);
  cudaError_t e = cudaSuccess;
  int rc = SIPG_OK;
  if (ctx->mapped) {
    const size_t nv = (size_t)(mesh->nx + 1) * (mesh->ny + 1) * (mesh->nz + 1) * 3;
    e = cudaMalloc(&ctx->dverts, sizeof(double) * nv);
    if (!e) e = cudaMemcpyAsync(ctx->dverts, mesh->vertices, sizeof(double) * nv, cudaMemcpyHostToDevice, ctx->st);
    if (e) rc = ctx->fail(SIPG_ERR_NOMEM, "vertices", e);
  }
  for (int op = 0; op < 2 && rc == SIPG_OK; ++op) rc = ctx->build_hierarchy(op);
  if (rc == SIPG_OK && ctx->mapped) {
    e = cudaStreamSynchronize(ctx->st);
    if (e) rc = ctx->fail(SIPG_ERR_CUDA, "vertices", e);
  }
  if (rc == SIPG_OK) {
    ctx->partials = dalloc<double>(kDotBlocks, &e, ctx->st);
    if (!e) ctx->dscal = dalloc<double>(16, &e, ctx->st);
    if (!e) ctx->dflag = dalloc<int>(4, &e, ctx->st);
    if (!e) e = cudaMallocHost(&ctx->hscal, 16 * sizeof(double));
    if (e) rc = ctx->fail(SIPG_ERR_NOMEM, "alloc scalars", e);
  }
  // the Poisson hierarchy's smoothers and coarse inverse are set up on first use
  if (rc != SIPG_OK) {
    fprintf(stderr, "sipg_create: %s\n", ctx->err.c_str());
    delete ctx;
    return rc;
  }
  *out = ctx;
  return SIPG_OK;
}

extern "C" int sipg_topology_tables(int nx, int ny, int nz, const unsigned char* active, const int* periodic,
                                    int* ncells, int* nbf, int* nbr, int* bface) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || !periodic || !ncells || !nbf) return SIPG_ERR_INVALID;
  if ((int64_t)nx * ny * nz > (int64_t)1 << 28) return SIPG_ERR_INVALID;
  const HostTopo t = host_topology(nx, ny, nz, active, periodic);
  *ncells = t.ncells;
  *nbf = t.nbf;
  if (nbr) std::copy(t.nbr.begin(), t.nbr.end(), nbr);
  if (bface) std::copy(t.bface.begin(), t.bface.end(), bface);
  return SIPG_OK;
}

extern "C" int sipg_coarsen_mask(int nx, int ny, int nz, const unsigned char* fine, unsigned char* coarse) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || nx % 2 || ny % 2 || nz % 2 || !fine || !coarse) return SIPG_ERR_INVALID;
  std::vector<unsigned char> f(fine, fine + (size_t)nx * ny * nz), c;
  if (!coarsen_mask(nx, ny, nz, f, &c)) return 0;
  std::copy(c.begin(), c.end(), coarse);
  return 1;
}

// Device bytes a context of this mesh and options allocates (no allocation).
extern "C" int sipg_estimate_bytes(const sipg_mesh_desc* mesh, const sipg_opts* opts_in, int64_t* bytes) {
  if (!mesh || !bytes) return SIPG_ERR_INVALID;
  sipg_opts o;
  sipg_default_opts(&o);
  if (opts_in) {
    o = *opts_in;
    sipg_opts d;
    sipg_default_opts(&d);
    if (o.coarse_max_dofs == 0) o.coarse_max_dofs = d.coarse_max_dofs;
    if (o.k_u == 0) o.k_u = d.k_u;
  }
  if (o.k_u < 2 || o.k_u > 5 || mesh->nx <= 0 || mesh->ny <= 0 || mesh->nz <= 0) return SIPG_ERR_INVALID;
  if (o.mg_cph != SIPG_MG_AUTO && o.mg_cph != SIPG_MG_DG && o.mg_cph != SIPG_MG_CPH) return SIPG_ERR_INVALID;
  o.mg_cph = resolved_mg_cph(o.mg_cph, mesh);
  sipg_ctx probe;
  probe.dry = true;
  probe.mesh = *mesh;
  probe.opts = o;
  probe.mapped = mesh->vertices != nullptr;
  probe.topo = mesh_topology(mesh);
  if (mesh->active) probe.mask.assign(mesh->active, mesh->active + (size_t)mesh->nx * mesh->ny * mesh->nz);
  probe.mesh.active = nullptr;
  probe.mesh.vertices = nullptr;
  for (int op = 0; op < 2; ++op) {
    int rc = probe.build_hierarchy(op);
    if (rc) return rc;
  }
  *bytes = probe.bytes + (int64_t)sizeof(double) * (kDotBlocks + 16) + 64;
  for (sipg::Hier& H : probe.hier)
    for (sipg::Level& L : H.L) {
      for (int p = 0; p < 2; ++p)
        for (int v = 0; v < 4; ++v) L.w[p][v] = nullptr;
    }
  return SIPG_OK;
}

extern "C" int sipg_level_plan(const sipg_mesh_desc* mesh, const sipg_opts* opts_in, int op, int max_levels,
                               int* nlevels, int* info) {
  if (!mesh || !nlevels || (op != SIPG_OP_VISCOUS && op != SIPG_OP_POISSON) || max_levels < 0) return SIPG_ERR_INVALID;
  sipg_opts o;
  sipg_default_opts(&o);
  if (opts_in) {
    o = *opts_in;
    sipg_opts d;
    sipg_default_opts(&d);
    if (o.coarse_max_dofs == 0) o.coarse_max_dofs = d.coarse_max_dofs;
    if (o.k_u == 0) o.k_u = d.k_u;
  }
  if (o.k_u < 2 || o.k_u > 5 || mesh->nx <= 0 || mesh->ny <= 0 || mesh->nz <= 0) return SIPG_ERR_INVALID;
  if (o.mg_cph != SIPG_MG_AUTO && o.mg_cph != SIPG_MG_DG && o.mg_cph != SIPG_MG_CPH) return SIPG_ERR_INVALID;
  o.mg_cph = resolved_mg_cph(o.mg_cph, mesh);
  sipg_ctx probe;
  probe.dry = true;
  probe.mesh = *mesh;
  probe.opts = o;
  probe.mapped = mesh->vertices != nullptr;
  probe.topo = mesh_topology(mesh);
  if (mesh->active) probe.mask.assign(mesh->active, mesh->active + (size_t)mesh->nx * mesh->ny * mesh->nz);
  probe.mesh.active = nullptr;
  probe.mesh.vertices = nullptr;
  int rc = probe.build_hierarchy(op);
  if (rc) return rc;
  const std::vector<Level>& L = probe.hier[op].L;
  *nlevels = (int)L.size();
  for (int l = 0; info && l < (int)L.size() && l < max_levels; ++l) {
    int* r = info + 6 * l;
    r[0] = L[l].g.nx;
    r[1] = L[l].g.ny;
    r[2] = L[l].g.nz;
    r[3] = L[l].k;
    r[4] = L[l].g.ncells;
    r[5] = (int)std::min<int64_t>(L[l].ndofs, 2147483647);
  }
  for (sipg::Hier& H : probe.hier)
    for (sipg::Level& Lv : H.L)
      for (int p = 0; p < 2; ++p)
        for (int v = 0; v < 4; ++v) Lv.w[p][v] = nullptr;
  return SIPG_OK;
}

extern "C" int sipg_destroy(sipg_ctx* ctx) {
  if (!ctx) return SIPG_ERR_INVALID;
  cudaStreamSynchronize(ctx->st);
  delete ctx;
  return SIPG_OK;
}

extern "C" const char* sipg_last_error(const sipg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int sipg_num_levels(const sipg_ctx* ctx, int op, int* n) {
  if (!ctx || (op != 0 && op != 1) || !n) return SIPG_ERR_INVALID;
  *n = (int)ctx->hier[op].L.size();
  return SIPG_OK;
}

extern "C" int sipg_level_info(const sipg_ctx* ctx, int op, int level, int* cells, int* degree, int64_t* ndofs) {
  if (!ctx || (op != 0 && op != 1)) return SIPG_ERR_INVALID;
  const Hier& H = ctx->hier[op];
  if (level < 0 || level >= (int)H.L.size()) return SIPG_ERR_INVALID;
  const Level& L = H.L[level];
  if (cells) { cells[0] = L.g.nx; cells[1] = L.g.ny; cells[2] = L.g.nz; }
  if (degree) *degree = L.k;
  if (ndofs) *ndofs = L.ndofs;
  return SIPG_OK;
}

// ------------------------------------------------------------ level pieces
template <typename T>
int sipg_ctx::level_apply(int op, int l, const T* x, T* y, double mass) {
  sipg_ctx* ctx = this;
  const Hier& H = hier[op];
  const Level& L = H.L[l];
  if (L.cg) {  // P^T A_DG P: gather, DG operator of the twin (same mesh and degree), sum the copies
    constexpr int p = sizeof(T) == 8 ? 0 : 1;
    T* a = static_cast<T*>(L.tdg[p][0]);
    T* b = static_cast<T*>(L.tdg[p][1]);
    const T* nc = nullptr;
    const T* nf = nullptr;
    if (op == SIPG_OP_VISCOUS) {
      if constexpr (sizeof(T) == 8) { nc = (const T*)L.nu_cell64; nf = (const T*)L.nu_face64; }
      else { nc = (const T*)L.nu_cell32; nf = (const T*)L.nu_face32; }
    }
    CK(launch_cg_map<T>(CG_GATHER, L.cgg, x, a, 1, st));
    CK((launch_apply<T>(L.n, H.ncomp, L.g, tabs[L.n], a, b, nc, nf, T(mass), 1, st)));
    CK(launch_cg_map<T>(CG_SCATTER_SUM, L.cgg, b, y, 1, st));
    return SIPG_OK;
  }
  if (mapped) {
    if constexpr (sizeof(T) == 8) {
      CK(launch_mapped_apply(L.n, H.ncomp, L.g, stabs[L.n], L.cmet64, L.fmet64, L.lam,
                             op == SIPG_OP_VISCOUS ? L.nu_cell64 : nullptr,
                             op == SIPG_OP_VISCOUS ? L.nu_face64 : nullptr, mass, (const double*)x, (double*)y, 1, st));
      return SIPG_OK;
    } else {
      CK(launch_mapped_apply_f32(L.n, H.ncomp, L.g, stabs[L.n], L.cmet32, L.fmet32, L.lam,
                                 op == SIPG_OP_VISCOUS ? L.nu_cell32 : nullptr,
                                 op == SIPG_OP_VISCOUS ? L.nu_face32 : nullptr, mass, (const float*)x, (float*)y, 1,
                                 st));
      return SIPG_OK;
    }
  }
  const T* nc = nullptr;
  const T* nf = nullptr;
  if (op == SIPG_OP_VISCOUS) {
    if constexpr (sizeof(T) == 8) { nc = (const T*)L.nu_cell64; nf = (const T*)L.nu_face64; }
    else { nc = (const T*)L.nu_cell32; nf = (const T*)L.nu_face32; }
  }
  CK((launch_apply<T>(L.n, H.ncomp, L.g, tabs[L.n], x, y, nc, nf, T(mass), 1, st)));
  return SIPG_OK;
}

int sipg_ctx::level_apply_ff(int op, int l, const double* x, double* y, double mass) {
  sipg_ctx* ctx = this;
  if (mapped) return fail(SIPG_ERR_INVALID, "trilinear cells: FP64 applies only");
  const Hier& H = hier[op];
  const Level& L = H.L[l];
  if (op == SIPG_OP_VISCOUS && !L.nu_cellff) return fail(SIPG_ERR_INVALID, "float-float apply on level 0 only");
  const float2* nc = op == SIPG_OP_VISCOUS ? L.nu_cellff : nullptr;
  const float2* nf = op == SIPG_OP_VISCOUS ? L.nu_faceff : nullptr;
  if (!L.xff) return fail(SIPG_ERR_INVALID, "float-float apply on level 0 only");
  CK(launch_split_ff_int(L.ndofs, x, L.xff, st));
  CK(launch_apply_ff(L.n, H.ncomp, L.g, tabs[L.n], L.xff, y, nc, nf, mass, 1, st));
  return SIPG_OK;
}

int sipg_ctx::krylov_apply(int op, const double* x, double* y, double mass) {
  return opts.krylov_arith == SIPG_F64_FF ? level_apply_ff(op, 0, x, y, mass)
                                          : level_apply<double>(op, 0, x, y, mass);
}

int sipg_ctx::dot(int64_t n, const double* a, const double* b, double* out_host) {
  sipg_ctx* ctx = this;
  CK(launch_dot(n, a, b, partials, dscal, st));
  CK(cudaMemcpyAsync(hscal, dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *out_host = hscal[0];
  return SIPG_OK;
}

// remove the mean (Euclidean projection onto the complement of constants)
int sipg_ctx::project_mean(int64_t n, double* v) {
  sipg_ctx* ctx = this;
  CK(launch_sum(n, v, partials, dscal + 1, st));
  CK(launch_add_const(n, dscal + 1, -1.0 / (double)n, v, st));
  return SIPG_OK;
}

// Largest eigenvalue of a symmetric tridiagonal matrix by bisection on the
// Sturm sequence count.
static double tridiag_lmax(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
      q = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= m) hi = mid; else lo = mid;
  }
  return hi;
}

int sipg_ctx::setup_level_smoother(int op, int l, double mass, bool estimate) {
  sipg_ctx* ctx = this;
  Hier& H = hier[op];
  Level& L = H.L[l];
  const double* nc = op == SIPG_OP_VISCOUS ? L.nu_cell64 : nullptr;
  const double* nf = op == SIPG_OP_VISCOUS ? L.nu_face64 : nullptr;
  if (mapped) {
    CK(launch_mapped_diagonal(L.n, H.ncomp, L.g, stabs[L.n], L.verts, L.lam, nc, nf, mass, L.diag64, st));
  } else if (L.cg) {  // sum over the copies of the cell and wall terms (jumps vanish)
    double* t = static_cast<double*>(L.tdg[0][0]);
    CK(launch_diagonal(L.n, H.ncomp, L.g, tabs[L.n], nc, nf, mass, t, st, false));
    CK(launch_cg_map<double>(CG_SCATTER_SUM, L.cgg, t, L.diag64, 1, st));
  } else {
    CK(launch_diagonal(L.n, H.ncomp, L.g, tabs[L.n], nc, nf, mass, L.diag64, st));
  }
  CK(launch_reciprocal(L.ndofs, L.diag64, L.dinv64, st));
  CK((launch_cast<double, float>(L.ndofs, L.dinv64, L.dinv32, st)));
  if (l + 1 == (int)H.L.size() || !estimate) return SIPG_OK;
  // Lanczos on D^-1/2 A D^-1/2 with level applies in the multigrid's arithmetic:
  // the Chebyshev smoother applies that operator, and the estimate needs a few
  // digits only (FP32 applies are 8x cheaper than FP64 ones on this GPU)
  const bool f32 = opts.mg_precision == SIPG_F32;
  float* w32 = (float*)L.w[1][2];
  float* t32 = (float*)L.w[1][3];
  double* q = (double*)L.w[0][0];
  double* qp = (double*)L.w[0][1];
  double* w = (double*)L.w[0][2];
  double* t = (double*)L.w[0][3];
  const int64_t n = L.ndofs;
  CK(launch_random(n, opts.seed + 7919ull * (uint64_t)(l + 1) + 104729ull * (uint64_t)op, q, st));
  if (H.singular && op == SIPG_OP_POISSON) { int rc = project_mean(n, q); if (rc) return rc; }
  double nrm;
  int rc = dot(n, q, q, &nrm);
  if (rc) return rc;
  CK(launch_scale(n, 1.0 / std::sqrt(nrm), q, q, st));
  CK(launch_fill<double>(n, 0.0, qp, st));
  std::vector<double> al, be;
  double beta = 0.0;
  // s = sqrt(dinv) once, kept in diag64 (the diagonal itself is not needed again
  // below the coarsest level)
  double* sd = L.diag64;
  CK((launch_cast<double, double>(n, L.dinv64, sd, st)));
  sqrt_inplace(n, sd);
  for (int j = 0; j < opts.lanczos_steps; ++j) {
    // w = s A (s q) - beta q_prev
    CK(launch_mul(n, sd, q, w, st));
    if (f32) {
      CK((launch_cast<double, float>(n, w, w32, st)));
      rc = level_apply<float>(op, l, w32, t32, mass);
      if (rc) return rc;
      CK((launch_cast<float, double>(n, t32, t, st)));
    } else {
      rc = level_apply<double>(op, l, w, t, mass);
      if (rc) return rc;
    }
    CK(launch_mul(n, sd, t, w, st));
    if (j > 0) CK(launch_add_scaled_f64(n, -beta, qp, w, st));
    double alpha;
    rc = dot(n, q, w, &alpha);
    if (rc) return rc;
    CK(launch_add_scaled_f64(n, -alpha, q, w, st));
    double bb;
    rc = dot(n, w, w, &bb);
    if (rc) return rc;
    al.push_back(alpha);
    beta = std::sqrt(bb);
    if (!(beta > 1e-300) || j + 1 == opts.lanczos_steps) break;
    be.push_back(beta);
    std::swap(q, qp);  // qp <- old q
    CK(launch_scale(n, 1.0 / beta, w, q, st));
  }
  be.resize(al.size() > 0 ? al.size() - 1 : 0);
  L.lmax = tridiag_lmax(al, be);
  // leave the work vectors zeroed for later use
  for (int v = 0; v < 4; ++v) CK(cudaMemsetAsync(L.w[0][v], 0, sizeof(double) * (size_t)n, st));
  for (int v = 2; v < 4; ++v) CK(cudaMemsetAsync(L.w[1][v], 0, sizeof(float) * (size_t)n, st));
  return SIPG_OK;
}

void sipg_ctx::sqrt_inplace(int64_t n, double* v) {
  // dinv >= 0 for an SPD operator; reuse the reciprocal + scale kernels is not
  // enough, so a dedicated elementwise sqrt lives in the vector helpers.
  launch_sqrt(n, v, st);
}

// Colouring of the cells of a (coarse) level for the column assembly of its DG
// operator: colour = (i mod c_x) + c_x ((j mod c_y) + c_y (k mod c_z)) with
// c_d = 3, or the extent n_d where n_d < 3 or where a periodic direction's extent
// is not a multiple of 3; two cells of one colour are then at least three cells
// apart along some direction, so their closed face neighbourhoods are disjoint.
// owner[colour * C + c'] = the cell of that colour in {c'} u N(c'), or -1.
int sipg_ctx::coarse_colouring(const LevelGeom& g, std::vector<int>* colour, std::vector<int>* owner, int* ncolours) {
  sipg_ctx* ctx = this;
  const int C = g.ncells;
  const int dims[3] = {g.nx, g.ny, g.nz};
  int cd[3];
  for (int d = 0; d < 3; ++d) {
    const bool per = g.nbr && mesh.periodic[d];
    cd[d] = dims[d] < 3 ? dims[d] : ((per && dims[d] % 3 != 0) ? dims[d] : 3);
  }
  std::vector<int> nbr((size_t)C * 6), cgrid;
  if (g.nbr) {
    cgrid.resize(C);
    CK(cudaMemcpy(nbr.data(), g.nbr, sizeof(int) * nbr.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(cgrid.data(), g.cgrid, sizeof(int) * C, cudaMemcpyDeviceToHost));
  }
  colour->assign(C, 0);
  for (int e = 0; e < C; ++e) {
    const int gi = g.nbr ? cgrid[e] : e;
    const int i = gi % g.nx, j = (gi / g.nx) % g.ny, k = gi / (g.nx * g.ny);
    (*colour)[e] = (i % cd[0]) + cd[0] * ((j % cd[1]) + cd[1] * (k % cd[2]));
    if (!g.nbr)
      for (int f = 0; f < 6; ++f) {
        const int d = f >> 1, s = f & 1;
        int ijk[3] = {i, j, k};
        ijk[d] += s ? 1 : -1;
        nbr[(size_t)e * 6 + f] = (ijk[d] < 0 || ijk[d] >= dims[d]) ? -1 : (ijk[2] * g.ny + ijk[1]) * g.nx + ijk[0];
      }
  }
  *ncolours = cd[0] * cd[1] * cd[2];
  if (*ncolours > C) {  // a grid with many removed cells: one colour per cell (the unit columns)
    for (int e = 0; e < C; ++e) (*colour)[e] = e;
    *ncolours = C;
  }
  owner->assign((size_t)*ncolours * C, -1);
  for (int e = 0; e < C; ++e) {
    const int col = (*colour)[e];
    (*owner)[(size_t)col * C + e] = e;
    for (int f = 0; f < 6; ++f) {
      const int nb = nbr[(size_t)e * 6 + f];
      if (nb >= 0) {
        int& o = (*owner)[(size_t)col * C + nb];
        if (o >= 0 && o != e) return fail(SIPG_ERR_STATE, "coarse colouring: overlapping neighbourhoods");
        o = e;
      }
    }
  }
  return SIPG_OK;
}

int sipg_ctx::setup_coarse(int op, double mass) {
  sipg_ctx* ctx = this;
  Hier& H = hier[op];
  Level& C = H.L.back();
  const int N = C.N;
  const int l = (int)H.L.size() - 1;
  if (H.singular && op == SIPG_OP_VISCOUS && mass == 0.0) return SIPG_OK;  // rigid modes: no inverse
  const double* nc = op == SIPG_OP_VISCOUS ? C.nu_cell64 : nullptr;
  const double* nf = op == SIPG_OP_VISCOUS ? C.nu_face64 : nullptr;
  if (!C.cg) {
    // columns of the DG operator by colouring (see coarse_colouring): one batched
    // apply of ncolours x (DoFs per cell) probe vectors instead of N unit vectors
    std::vector<int> colour, owner;
    int ncol = 0;
    int rc = coarse_colouring(C.g, &colour, &owner, &ncol);
    if (rc) return rc;
    const int dpc = H.ncomp * C.n * C.n * C.n;
    const int nb = ncol * dpc;
    int *dcol = nullptr, *down = nullptr;
    CK(cudaMalloc(&dcol, sizeof(int) * colour.size()));
    cudaError_t ce = cudaMalloc(&down, sizeof(int) * owner.size());
    if (!ce) ce = cudaMemcpyAsync(dcol, colour.data(), sizeof(int) * colour.size(), cudaMemcpyHostToDevice, st);
    if (!ce) ce = cudaMemcpyAsync(down, owner.data(), sizeof(int) * owner.size(), cudaMemcpyHostToDevice, st);
    if (!ce) ce = launch_colour_probes(N, dpc, nb, dcol, C.Atmp, st);
    if (!ce)
      ce = mapped ? launch_mapped_apply(C.n, H.ncomp, C.g, stabs[C.n], C.cmet64, C.fmet64, C.lam, nc, nf, mass,
                                        C.Atmp, C.Ainv, nb, st)
                  : launch_apply<double>(C.n, H.ncomp, C.g, tabs[C.n], C.Atmp, C.Ainv, nc, nf, mass, nb, st);
    if (!ce) ce = cudaMemsetAsync(C.Atmp, 0, sizeof(double) * (size_t)N * N, st);
    if (!ce) ce = launch_colour_scatter(N, C.g.ncells, dpc, nb, down, C.Ainv, C.Atmp, st);
    if (!ce) ce = cudaMemcpyAsync(C.Ainv, C.Atmp, sizeof(double) * (size_t)N * N, cudaMemcpyDeviceToDevice, st);
    if (!ce) ce = cudaStreamSynchronize(st);
    cudaFree(dcol);
    cudaFree(down);
    CK(ce);
  } else {
    // continuous coarse level: columns P^T A_DG P e_j in chunks of columns (gather,
    // batched DG apply, batched sum over copies)
    CK(launch_unit_columns(N, 0, N, C.Atmp, st));
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(N, (int64_t)(64 << 20) / (16 * C.ndg)));
    double *ga = nullptr, *gb = nullptr;
    CK(cudaMalloc(&ga, sizeof(double) * (size_t)C.ndg * chunk));
    CK(cudaMalloc(&gb, sizeof(double) * (size_t)C.ndg * chunk));
    cudaError_t ce = cudaSuccess;
    for (int j0 = 0; j0 < N && ce == cudaSuccess; j0 += chunk) {
      const int nb = std::min(chunk, N - j0);
      ce = launch_cg_map<double>(CG_GATHER, C.cgg, C.Atmp + (size_t)j0 * N, ga, nb, st);
      if (ce == cudaSuccess)
        ce = launch_apply<double>(C.n, H.ncomp, C.g, tabs[C.n], ga, gb, nc, nf, mass, nb, st);
      if (ce == cudaSuccess) ce = launch_cg_map<double>(CG_SCATTER_SUM, C.cgg, gb, C.Ainv + (size_t)j0 * N, nb, st);
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    cudaFree(ga);
    cudaFree(gb);
    CK(ce);
  }
  (void)l;
  // column j of A is stored contiguously: that is A^T row-major = A (symmetric)
  if (H.singular && op == SIPG_OP_POISSON && mass == 0.0) {
    // constant null space: A + c 1 1^T is SPD and solves A x = b for mean-free b
    // scale c from the mean diagonal, so that c 1^T 1 is of the operator's size
    CK(launch_sum(N, C.diag64, partials, dscal + 2, st));
    CK(cudaMemcpyAsync(hscal, dscal + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double mean_diag = hscal[0] / N;
    CK(launch_add_rank1(N, mean_diag / N, C.Ainv, st));
  }
  // Gauss-Jordan inverse in float-float storage (48-bit significands, the FP32
  // pipe instead of the 75x slower FP64 one), ping-pong between the two
  // buffers, converted back to binary64 once at the end
  CK(launch_to_ff_inplace((int64_t)N * N, C.Ainv, st));
  float2* A = reinterpret_cast<float2*>(C.Ainv);
  float2* B = reinterpret_cast<float2*>(C.Atmp);
  // blocks of 16 pivots: three launches per block instead of one per pivot
  float2* Pinv = reinterpret_cast<float2*>(C.gjw);
  float2* R = Pinv + 256;
  for (int k0 = 0; k0 < N; k0 += 16) {
    CK(launch_gj_block(N, k0, std::min(16, N - k0), A, B, Pinv, R, st));
    std::swap(A, B);
  }
  if (A != reinterpret_cast<float2*>(C.Ainv))
    CK(cudaMemcpyAsync(C.Ainv, A, sizeof(double) * (size_t)N * N, cudaMemcpyDeviceToDevice, st));
  CK(launch_from_ff_inplace((int64_t)N * N, C.Ainv, st));
  return SIPG_OK;
}

int sipg_ctx::ensure_setup(int op) {
  if (hier[op].ready) return SIPG_OK;
  if (op == SIPG_OP_VISCOUS && !have_nu) return fail(SIPG_ERR_STATE, "set the viscosity first");
  return setup_operator(op, hier[op].setup_mass);
}

int sipg_ctx::setup_operator(int op, double mass) {
  sipg_ctx* ctx = this;
  Hier& H = hier[op];
  const int lag = opts.mg_setup_lag > 1 ? opts.mg_setup_lag : 1;
  const bool full = !H.have_full || H.full_mass != mass || H.updates_since_full + 1 >= lag;
  for (size_t l = 0; l < H.L.size(); ++l) {
    int rc = setup_level_smoother(op, (int)l, mass, full);
    if (rc) return rc;
  }
  if (full) {
    int rc = setup_coarse(op, mass);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(st));
  H.setup_mass = mass;
  H.ready = true;
  H.updates_since_full = full ? 0 : H.updates_since_full + 1;
  H.have_full = true;
  H.full_mass = mass;
  return SIPG_OK;
}

// ------------------------------------------------------------ viscosity
int sipg_ctx::parse_rheology(const sipg_rheology* rh, const double* u_lin, RheologyDev* out) {
  RheologyDev& r = *out;
  r = RheologyDev{};
  r.law = rh->law;
  switch (rh->law) {
    case SIPG_LAW_CONSTANT:
      if (!(rh->nu > 0)) return fail(SIPG_ERR_INVALID, "constant viscosity must be positive");
      r.nu = rh->nu;
      break;
    case SIPG_LAW_ANALYTIC:
      break;
    case SIPG_LAW_SINKER:
      if (rh->n_spheres < 0 || rh->n_spheres > 64 || (rh->n_spheres > 0 && !rh->centers))
        return fail(SIPG_ERR_INVALID, "sinker: 0..64 spheres with a host centre array");
      if (!(rh->nu_max > 0) || !(rh->nu_matrix > 0)) return fail(SIPG_ERR_INVALID, "sinker viscosities must be positive");
      r.n_spheres = rh->n_spheres;
      std::memcpy(r.centers, rh->centers, sizeof(double) * 3 * rh->n_spheres);
      r.radius = rh->radius;
      r.nu_max = rh->nu_max;
      r.nu_matrix = rh->nu_matrix;
      break;
    case SIPG_LAW_CARREAU:
      if (!u_lin) return fail(SIPG_ERR_INVALID, "Carreau-Yasuda viscosity needs the linearization velocity");
      if (!(rh->eta0 > 0) || !(rh->eta_inf >= 0) || !(rh->a > 0))
        return fail(SIPG_ERR_INVALID, "Carreau-Yasuda parameters out of range");
      r.eta0 = rh->eta0; r.eta_inf = rh->eta_inf; r.kappa = rh->kappa; r.lambda = rh->lambda;
      r.a = rh->a; r.b = rh->b;
      break;
    default:
      return fail(SIPG_ERR_INVALID, "unknown viscosity law");
  }
  return SIPG_OK;
}

// nu at the quadrature points of every level of the viscous hierarchy (no
// smoother or coarse setup; the hierarchy is marked stale)
int sipg_ctx::eval_viscosity(const RheologyDev& r, const double* u_lin) {
  Hier& H = hier[SIPG_OP_VISCOUS];
  std::vector<Level>& DL = H.cph ? H.T : H.L;  // the DG sequence holds the viscosity storage
  for (size_t l = 0; l < DL.size(); ++l) {
    Level& L = DL[l];
    const double* u = nullptr;
    if (r.law == SIPG_LAW_CARREAU) {
      if (l == 0) {
        u = u_lin;
      } else {
        Level& F = DL[l - 1];
        const double* uf = l == 1 ? u_lin : F.ulin;
        cudaError_t e = F.next_kind == 1
                            ? launch_p_interp_down(F.n, L.n, 3, L.g.ncells, F.interp, uf, L.ulin, st)
                            : launch_h_interp_down(L.n, 3, F.g, L.g, F.interp, F.child, uf, L.ulin, st);
        if (e) return fail(SIPG_ERR_CUDA, "interpolate linearization velocity", e);
        u = L.ulin;
      }
    }
    cudaError_t e;
    if (r.law == SIPG_LAW_SINKER && l > 0) {
      // cellwise-constant field: carried down by the transfer of piecewise constants
      const Level& F = DL[l - 1];
      e = launch_cell_nu_transfer(F.g, L.g, F.next_kind, F.n, L.n, F.nu_cell64, L.nu_cell64, L.nu_face64, st);
    } else if (mapped) {
      e = launch_mapped_viscosity(L.n, L.g, stabs[L.n], L.verts, r, u, L.nu_cell64, L.nu_face64, st);
    } else {
      e = launch_viscosity(L.n, L.g, tabs[L.n], r, u, L.nu_cell64, L.nu_face64, st);
    }
    if (e) return fail(SIPG_ERR_CUDA, "viscosity kernel", e);
    const int64_t n3 = (int64_t)L.n * L.n * L.n, n2 = (int64_t)L.n * L.n;
    e = launch_cast<double, float>(L.g.ncells * n3, L.nu_cell64, L.nu_cell32, st);
    if (!e) e = launch_cast<double, float>(L.g.ncells * 6 * n2, L.nu_face64, L.nu_face32, st);
    if (!e && L.nu_cellff) e = launch_split_ff(L.g.ncells * n3, L.nu_cell64, L.nu_cellff, st);
    if (!e && L.nu_faceff) e = launch_split_ff(L.g.ncells * 6 * n2, L.nu_face64, L.nu_faceff, st);
    if (e) return fail(SIPG_ERR_CUDA, "viscosity cast", e);
  }
  have_nu = true;
  H.ready = false;
  return SIPG_OK;
}

extern "C" int sipg_set_viscosity(sipg_ctx* ctx, const sipg_rheology* rh, const double* u_lin) {
  if (!ctx || !rh) return SIPG_ERR_INVALID;
  RheologyDev r;
  int rc = ctx->parse_rheology(rh, u_lin, &r);
  if (rc) return rc;
  if ((rc = ctx->eval_viscosity(r, u_lin))) return rc;
  return ctx->setup_operator(SIPG_OP_VISCOUS, 0.0);
}

// ------------------------------------------------------------ apply
static int check_op(sipg_ctx* ctx, int op) {
  if (op != SIPG_OP_VISCOUS && op != SIPG_OP_POISSON) return ctx->fail(SIPG_ERR_INVALID, "unknown operator");
  if (op == SIPG_OP_VISCOUS && !ctx->have_nu) return ctx->fail(SIPG_ERR_STATE, "set the viscosity first");
  return SIPG_OK;
}

extern "C" int sipg_level_apply(sipg_ctx* ctx, int op, int level, int prec, const void* x, void* y, double mass) {
  if (!ctx) return SIPG_ERR_INVALID;
  int rc = check_op(ctx, op);
  if (rc) return rc;
  if (level < 0 || level >= (int)ctx->hier[op].L.size() || !x || !y || x == y)
    return ctx->fail(SIPG_ERR_INVALID, "bad level or buffers");
  if (prec == SIPG_F64) return ctx->level_apply<double>(op, level, (const double*)x, (double*)y, mass);
  if (prec == SIPG_F32) return ctx->level_apply<float>(op, level, (const float*)x, (float*)y, mass);
  if (prec == SIPG_F64_FF) return ctx->level_apply_ff(op, level, (const double*)x, (double*)y, mass);
  return ctx->fail(SIPG_ERR_INVALID, "bad precision");
}

extern "C" int sipg_apply(sipg_ctx* ctx, int op, int prec, const void* x, void* y, double mass) {
  return sipg_level_apply(ctx, op, 0, prec, x, y, mass);
}

int sipg_ctx::mass_apply(int op, int prec, const void* x, void* y, double coeff, bool inverse) {
  sipg_ctx* ctx = this;
  if (op != SIPG_OP_VISCOUS && op != SIPG_OP_POISSON) return fail(SIPG_ERR_INVALID, "unknown operator");
  if (prec != SIPG_F64 && prec != SIPG_F32 && prec != SIPG_F64_FF) return fail(SIPG_ERR_INVALID, "unknown arithmetic");
  if (!x || !y) return fail(SIPG_ERR_INVALID, "null vector");
  if (!std::isfinite(coeff) || (inverse && coeff == 0.0)) return fail(SIPG_ERR_INVALID, "mass coefficient");
  const Hier& H = hier[op];
  const Level& L = H.L[0];
  if (mapped) {  // trilinear cells: w det J per point (FP64; S^-1 diag S^-T for the inverse)
    if (prec == SIPG_F32) return fail(SIPG_ERR_INVALID, "trilinear cells: FP64 mass operators");
    CK(launch_mapped_mass(L.n, H.ncomp, L.g, stabs[L.n], L.verts, coeff, inverse, (const double*)x, (double*)y, st));
    return SIPG_OK;
  }
  const double detJ = L.g.h[0] * L.g.h[1] * L.g.h[2];
  const double scale = inverse ? 1.0 / (coeff * detJ) : coeff * detJ;
  CK(launch_cell_mass(L.n, H.ncomp, L.g.ncells, tabs[L.n], prec, inverse, scale, x, y, st));
  return SIPG_OK;
}

extern "C" int sipg_ff_convert(sipg_ctx* ctx, const double* x, float* hilo, double* back, int64_t n) {
  if (!ctx || n < 0 || (n > 0 && (!x || !hilo || !back))) return SIPG_ERR_INVALID;
  CK(launch_ff_convert(n, x, reinterpret_cast<float2*>(hilo), back, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return SIPG_OK;
}

extern "C" int sipg_mass_apply(sipg_ctx* ctx, int op, int prec, const void* x, void* y, double coeff) {
  if (!ctx) return SIPG_ERR_INVALID;
  return ctx->mass_apply(op, prec, x, y, coeff, false);
}

extern "C" int sipg_inverse_mass_apply(sipg_ctx* ctx, int op, int prec, const void* x, void* y, double coeff) {
  if (!ctx) return SIPG_ERR_INVALID;
  return ctx->mass_apply(op, prec, x, y, coeff, true);
}

extern "C" int sipg_apply_host(sipg_ctx* ctx, int op, const double* xh, double* yh, double mass) {
  if (!ctx || !xh || !yh) return SIPG_ERR_INVALID;
  int rc = check_op(ctx, op);
  if (rc) return rc;
  const int64_t n = ctx->hier[op].L[0].ndofs;
  if (ctx->host_n < n) {
    cudaFree(ctx->host_x);
    cudaFree(ctx->host_y);
    ctx->host_x = ctx->host_y = nullptr;
    ctx->host_n = 0;
    CK(cudaMalloc(&ctx->host_x, sizeof(double) * n));
    CK(cudaMalloc(&ctx->host_y, sizeof(double) * n));
    ctx->host_n = n;
  }
  CK(cudaMemcpyAsync(ctx->host_x, xh, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st));
  rc = ctx->krylov_apply(op, ctx->host_x, ctx->host_y, mass);
  if (rc) return rc;
  CK(cudaMemcpyAsync(yh, ctx->host_y, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return SIPG_OK;
}

template int sipg_ctx::level_apply<double>(int, int, const double*, double*, double);
template int sipg_ctx::level_apply<float>(int, int, const float*, float*, double);
