// Continuous-batching solve server.
//
// Requests (a box mesh, a degree, a viscosity field, a right-hand side, a
// tolerance) are queued by sipg_server_submit and served by one worker thread:
//  * admission: a queued request starts when a slot is free and the device
//    bytes of its context (sipg_estimate_bytes) fit the HBM budget; contexts
//    are cached per (mesh, degree) and reused, so finishing a request frees
//    its slot and memory without a device-wide synchronisation;
//  * rounds: every active request advances by one preconditioned CG
//    iteration per round, with all CG scalars kept on the device. The
//    fine-level operator applies of all active requests of one degree run in
//    ONE persistent launch (apply_multi_kernel: CTAs stride over a tile list
//    that spans the requests); dot products, vector updates and the
//    multigrid V-cycle of each request run on that request's own stream, so
//    the requests' work overlaps on the device;
//  * requests that arrive while others are running join at the next round
//    (continuous batching); a finished request leaves at the end of a round.
// Each request's arithmetic is the same kernel sequence as a solve on its own
// (the batched launch computes every cell with the same code as the single
// launch), so its result does not depend on the mix.
// Right-hand sides: b = A u* for a seeded u* (the error against u* is then
// reported), the buoyancy load M f of the request's spheres, or the caller's
// own vector from host or device memory.
#include "../../include/sipg.h"
#include "ctx.h"
#include "kernels.cuh"
#include "operator.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <type_traits>
#include <vector>

using namespace sipg;

namespace {

using Clock = std::chrono::steady_clock;

// device CG scalars of one request: [0] rz, [1] pq, [2] rr, [3] rz_new,
// [4] bnorm2, [5] breakdown flag
__global__ void cg_step_x_r(int64_t n, const double* __restrict__ sc, const double* __restrict__ p,
                            const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r) {
  const double pq = sc[1];
  if (!(pq > 0.0) || !isfinite(pq)) return;  // breakdown: leave x, r (flag set by cg_check)
  const double alpha = sc[0] / pq;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
  }
}

__global__ void cg_step_p(int64_t n, const double* __restrict__ sc, const double* __restrict__ z,
                          double* __restrict__ p) {
  const double beta = sc[0] != 0.0 ? sc[3] / sc[0] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

__global__ void cg_check(double* sc) {
  const double pq = sc[1];
  if (!(pq > 0.0) || !isfinite(pq)) sc[5] = 1.0;
}

__global__ void cg_rotate(double* sc) { sc[0] = sc[3]; }

inline int vec_blocks(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 8); }

struct Request {
  uint64_t id = 0;
  sipg_request spec{};
  sipg_rheology rh{};
  std::vector<double> centers;
  std::vector<double> b_host;  // rhs HOST: the caller's b, copied by submit
  bool keep_solution = false;
  // runtime
  sipg_ctx* ctx = nullptr;
  int64_t n = 0, bytes = 0;
  double *ustar = nullptr, *b = nullptr, *x = nullptr, *sc = nullptr;
  double* hsc = nullptr;  // pinned: rr, flag
  cudaEvent_t ev_ready = nullptr, ev_rr = nullptr;
  int iters = 0;
  int replacements = 0;  // restarts from the true residual (see confirm_or_restart)
  double bnorm = 0.0;
  Clock::time_point t_submit, t_admit, t_done;
  sipg_result result{};
  std::vector<double> solution;
  bool done = false;
};

struct ContextEntry {
  sipg_ctx* ctx;
  int nc, k;
  int64_t bytes;
  bool busy;
  // request-side buffers owned with the context (b, u*, x, scalars)
  double *ustar, *b, *x, *sc;
  double* hsc;
  cudaEvent_t ev_ready, ev_rr;
};

}  // namespace

struct sipg_server {
  sipg_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::deque<std::unique_ptr<Request>> queue;
  std::vector<Request*> active;
  std::map<uint64_t, std::unique_ptr<Request>> finished;
  std::vector<ContextEntry> pool;
  uint64_t next_id = 1;
  int64_t used_bytes = 0;
  int pending = 0;  // queued + active
  bool stop = false;
  bool failed = false;
  std::string err;
  std::thread worker;
  cudaStream_t sched = nullptr;
  cudaEvent_t ev_applied = nullptr;
  int device = 0;
  // batched-apply tables per degree (device copies rebuilt every round); the
  // descriptors are ApplyDesc<double, ff> or ApplyDesc<double, double>
  std::vector<unsigned char> h_desc;
  std::vector<int2> h_tiles;
  void* d_desc = nullptr;
  int2* d_tiles = nullptr;
  size_t d_desc_cap = 0, d_tiles_cap = 0;

  void run();
  bool admit_one(std::unique_ptr<Request>& rq);
  int start_request(Request* r);
  int round();
  template <typename TN>
  int batched_apply(const std::map<int, std::vector<Request*>>& by_k);
  int finish(Request* r);
  int confirm_or_restart(Request* r, bool* restarted);
  int acquire_context(int nc, int k, int64_t need, ContextEntry** out);
  void release_entry(ContextEntry& c);
  void set_error(const std::string& m) {
    failed = true;
    err = m;
  }
};

namespace {

sipg_mesh_desc box_mesh(int nc) {
  sipg_mesh_desc m{};
  m.nx = m.ny = m.nz = nc;
  m.lx = m.ly = m.lz = 1.0;
  for (int i = 0; i < 6; ++i) {
    m.bc_velocity[i] = SIPG_BC_DIRICHLET;
    m.bc_pressure[i] = SIPG_BC_NEUMANN;
  }
  return m;
}

}  // namespace

// Frees the request-side buffers, the context and its stream of a pool entry.
void sipg_server::release_entry(ContextEntry& c) {
  cudaFree(c.ustar);
  cudaFree(c.b);
  cudaFree(c.x);
  cudaFree(c.sc);
  if (c.hsc) cudaFreeHost(c.hsc);
  if (c.ev_ready) cudaEventDestroy(c.ev_ready);
  if (c.ev_rr) cudaEventDestroy(c.ev_rr);
  if (c.ctx) {
    cudaStream_t st = c.ctx->st;
    sipg_destroy(c.ctx);
    cudaStreamDestroy(st);
  }
  c = ContextEntry{};
}

// A context for an nc^3 mesh of degree k: an idle cached one, or a new one
// after evicting idle contexts of other shapes until `need` bytes fit.
// Returns SIPG_OK (*out set), SIPG_PENDING (the budget is held by busy
// contexts: retry after a round) or an error (nothing is left allocated).
int sipg_server::acquire_context(int nc, int k, int64_t need, ContextEntry** out) {
  *out = nullptr;
  for (ContextEntry& c : pool)
    if (!c.busy && c.nc == nc && c.k == k) {
      c.busy = true;
      *out = &c;
      return SIPG_OK;
    }
  while (used_bytes + need > (int64_t)opts.hbm_budget_bytes) {
    auto it = std::find_if(pool.begin(), pool.end(), [](const ContextEntry& c) { return !c.busy; });
    if (it == pool.end()) return SIPG_PENDING;
    used_bytes -= it->bytes;
    release_entry(*it);
    pool.erase(it);
  }
  sipg_opts o;
  sipg_default_opts(&o);
  o.k_u = k;
  o.mg_precision = opts.mg_precision;
  o.cheb_degree = opts.cheb_degree > 0 ? opts.cheb_degree : 3;
  o.krylov_arith = opts.krylov_arith;
  ContextEntry c{};
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SIPG_ERR_CUDA;
  sipg_mesh_desc m = box_mesh(nc);
  const int rc = sipg_create(&m, &o, st, &c.ctx);
  if (rc != SIPG_OK) {
    cudaStreamDestroy(st);
    return rc;
  }
  c.nc = nc;
  c.k = k;
  c.bytes = need;
  c.busy = true;
  const int64_t n = c.ctx->hier[SIPG_OP_VISCOUS].L[0].ndofs;
  const bool mem = cudaMalloc(&c.ustar, sizeof(double) * n) == cudaSuccess &&
                   cudaMalloc(&c.b, sizeof(double) * n) == cudaSuccess &&
                   cudaMalloc(&c.x, sizeof(double) * n) == cudaSuccess &&
                   cudaMalloc(&c.sc, sizeof(double) * 16) == cudaSuccess;
  const bool ok = mem && cudaMallocHost(&c.hsc, sizeof(double) * 4) == cudaSuccess &&
                  cudaEventCreateWithFlags(&c.ev_ready, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&c.ev_rr, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();  // clear a sticky-free allocation error
    release_entry(c);
    return mem ? SIPG_ERR_CUDA : SIPG_ERR_NOMEM;
  }
  used_bytes += need;
  pool.push_back(c);
  *out = &pool.back();
  return SIPG_OK;
}

bool sipg_server::admit_one(std::unique_ptr<Request>& rq) {
  sipg_mesh_desc m = box_mesh(rq->spec.n_cells);
  sipg_opts o;
  sipg_default_opts(&o);
  o.k_u = rq->spec.k_u;
  o.mg_precision = opts.mg_precision;
  o.cheb_degree = opts.cheb_degree > 0 ? opts.cheb_degree : 3;
  o.krylov_arith = opts.krylov_arith;
  int64_t need = 0;
  const int erc = sipg_estimate_bytes(&m, &o, &need);
  if (erc != SIPG_OK) {  // a mesh the library refuses: fail the request
    rq->result.status = erc;
    rq->done = true;
    return true;
  }
  const int64_t n = (int64_t)rq->spec.n_cells * rq->spec.n_cells * rq->spec.n_cells * 3 * (rq->spec.k_u + 1) *
                    (rq->spec.k_u + 1) * (rq->spec.k_u + 1);
  need += 3 * 8 * n + 256;  // u*, b, x of the request
  if (need > (int64_t)opts.hbm_budget_bytes) {  // can never fit: reject now
    rq->result.status = SIPG_ERR_NOMEM;
    rq->done = true;
    return true;
  }
  ContextEntry* c = nullptr;
  const int rc = acquire_context(rq->spec.n_cells, rq->spec.k_u, need, &c);
  if (rc == SIPG_PENDING) return false;  // wait for memory held by running requests
  if (rc != SIPG_OK) {                    // the context could not be built: fail the request
    rq->result.status = rc;
    rq->done = true;
    return true;
  }
  Request* r = rq.get();
  r->ctx = c->ctx;
  r->ustar = c->ustar;
  r->b = c->b;
  r->x = c->x;
  r->sc = c->sc;
  r->hsc = c->hsc;
  r->ev_ready = c->ev_ready;
  r->ev_rr = c->ev_rr;
  r->bytes = need;
  r->n = c->ctx->hier[SIPG_OP_VISCOUS].L[0].ndofs;
  r->t_admit = Clock::now();
  return true;
}

// nodal interpolant of -e_z chi(x) (chi: inside any sphere, |x - c| <= r) on the
// box level g, velocity layout ((cell*3 + c)*n + iz)*n^2 + iy*n + ix
struct SphereSet {
  int count;
  double r2;
  double c[3 * 64];
};
struct NodeSet {
  double x[kMaxN];
};
__global__ void buoyancy_kernel(LevelGeom g, int n, NodeSet nodes, SphereSet sp, double* __restrict__ f) {
  const int n3 = n * n * n;
  const int64_t total = (int64_t)g.ncells * 3 * n3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / (3 * n3);
    const int r = (int)(i - e * 3 * n3);
    const int comp = r / n3, q = r - comp * n3;
    if (comp != 2) {
      f[i] = 0.0;
      continue;
    }
    const int ix = q % n, iy = (q / n) % n, iz = q / (n * n);
    int ijk[3];
    cell_ijk(g, (int)e, ijk);
    const double p[3] = {g.x0[0] + (ijk[0] + nodes.x[ix]) * g.h[0], g.x0[1] + (ijk[1] + nodes.x[iy]) * g.h[1],
                         g.x0[2] + (ijk[2] + nodes.x[iz]) * g.h[2]};
    bool inside = false;
    for (int s = 0; s < sp.count; ++s) {
      const double dx = p[0] - sp.c[3 * s], dy = p[1] - sp.c[3 * s + 1], dz = p[2] - sp.c[3 * s + 2];
      inside |= dx * dx + dy * dy + dz * dz <= sp.r2;
    }
    f[i] = inside ? -1.0 : 0.0;
  }
}

// viscosity, right-hand side, and the first CG step, on the request's stream
int sipg_server::start_request(Request* r) {
  sipg_ctx* ctx = r->ctx;
  sipg_rheology rh = r->rh;
  rh.centers = r->centers.data();
  int rc = sipg_set_viscosity(ctx, &rh, nullptr);
  if (rc) return rc;
  cudaStream_t st = ctx->st;
  Hier& H = ctx->hier[SIPG_OP_VISCOUS];
  double *rr = H.cg[0], *z = H.cg[1], *p = H.cg[2];
  const int64_t n = r->n;
  switch (r->spec.rhs) {
    case SIPG_RHS_MANUFACTURED:
      if (launch_random(n, r->spec.seed, r->ustar, st)) return SIPG_ERR_CUDA;
      rc = ctx->krylov_apply(SIPG_OP_VISCOUS, r->ustar, r->b, 0.0);
      if (rc) return rc;
      break;
    case SIPG_RHS_BUOYANCY: {
      const Level& L0 = H.L[0];
      NodeSet nodes{};
      for (int i = 0; i < L0.n; ++i) nodes.x[i] = ctx->tabs[L0.n].gll[i];
      SphereSet sp{};
      sp.count = r->rh.law == SIPG_LAW_SINKER ? r->rh.n_spheres : 0;
      sp.r2 = r->rh.radius * r->rh.radius;
      for (int i = 0; i < 3 * sp.count; ++i) sp.c[i] = r->centers[i];
      buoyancy_kernel<<<vec_blocks(n), 256, 0, st>>>(L0.g, L0.n, nodes, sp, r->ustar);
      if (cudaGetLastError()) return SIPG_ERR_CUDA;
      rc = ctx->mass_apply(SIPG_OP_VISCOUS, SIPG_F64, r->ustar, r->b, 1.0, false);
      if (rc) return rc;
      break;
    }
    case SIPG_RHS_HOST:
      if (cudaMemcpyAsync(r->b, r->b_host.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st))
        return SIPG_ERR_CUDA;
      break;
    default:  // SIPG_RHS_DEVICE
      if (cudaMemcpyAsync(r->b, r->spec.b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st)) return SIPG_ERR_CUDA;
      break;
  }
  if (cudaMemsetAsync(r->x, 0, sizeof(double) * n, st)) return SIPG_ERR_CUDA;
  if (cudaMemsetAsync(r->sc, 0, sizeof(double) * 16, st)) return SIPG_ERR_CUDA;
  if (cudaMemcpyAsync(rr, r->b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st)) return SIPG_ERR_CUDA;
  if (launch_dot(n, r->b, r->b, ctx->partials, r->sc + 4, st)) return SIPG_ERR_CUDA;
  if (cudaMemcpyAsync(r->hsc + 2, r->sc + 4, sizeof(double), cudaMemcpyDeviceToHost, st)) return SIPG_ERR_CUDA;
  rc = ctx->precondition(SIPG_OP_VISCOUS, SIPG_PRECOND_MG, rr, z, 0.0);
  if (rc) return rc;
  if (cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st)) return SIPG_ERR_CUDA;
  if (launch_dot(n, rr, z, ctx->partials, r->sc + 0, st)) return SIPG_ERR_CUDA;
  if (cudaStreamSynchronize(st)) return SIPG_ERR_CUDA;
  r->bnorm = std::sqrt(r->hsc[2]);
  std::vector<double>().swap(r->b_host);  // copied: release the host copy
  return SIPG_OK;
}

// q_i = A_i p_i of every active request: one persistent launch per degree
// present. TN is the viscosity type of the operator (ff: float-float, double:
// native FP64).
template <typename TN>
int sipg_server::batched_apply(const std::map<int, std::vector<Request*>>& by_k) {
  using Desc = ApplyDesc<double, TN>;
  size_t ndesc = 0, ntile = 0;
  for (auto& kv : by_k)
    for (Request* r : kv.second) {
      const int cpb = op_cells_per_cta(kv.first + 1, 3);
      ntile += (r->ctx->hier[SIPG_OP_VISCOUS].L[0].g.ncells + cpb - 1) / cpb;
      ++ndesc;
    }
  if (ndesc * sizeof(Desc) > d_desc_cap) {
    cudaFree(d_desc);
    d_desc = nullptr;
    d_desc_cap = std::max<size_t>(ndesc * sizeof(Desc), 2 * d_desc_cap);
    if (cudaMalloc(&d_desc, d_desc_cap)) {
      d_desc_cap = 0;
      return SIPG_ERR_NOMEM;
    }
  }
  if (ntile > d_tiles_cap) {
    cudaFree(d_tiles);
    d_tiles = nullptr;
    d_tiles_cap = std::max<size_t>(ntile, 2 * d_tiles_cap);
    if (cudaMalloc(&d_tiles, sizeof(int2) * d_tiles_cap)) {
      d_tiles_cap = 0;
      return SIPG_ERR_NOMEM;
    }
  }
  std::vector<Desc> descs;
  h_tiles.clear();
  std::vector<std::pair<int, std::pair<size_t, size_t>>> groups;  // degree, tile range
  for (auto& kv : by_k) {
    const size_t t0 = h_tiles.size();
    for (Request* r : kv.second) {
      const Level& L = r->ctx->hier[SIPG_OP_VISCOUS].L[0];
      Desc d{};
      d.g = L.g;
      d.x = r->ctx->hier[SIPG_OP_VISCOUS].cg[2];  // p
      d.y = r->ctx->hier[SIPG_OP_VISCOUS].cg[3];  // q
      if constexpr (std::is_same<TN, ff>::value) {
        d.nu_cell = reinterpret_cast<const ff*>(L.nu_cellff);
        d.nu_face = reinterpret_cast<const ff*>(L.nu_faceff);
      } else {
        d.nu_cell = L.nu_cell64;
        d.nu_face = L.nu_face64;
      }
      d.lc = level_consts<TN>(L.g, kv.first + 1, 0.0);
      const int di = (int)descs.size();
      descs.push_back(d);
      const int cpb = op_cells_per_cta(kv.first + 1, 3);
      for (int c0 = 0; c0 < L.g.ncells; c0 += cpb) h_tiles.push_back(make_int2(di, c0));
    }
    groups.push_back({kv.first, {t0, h_tiles.size() - t0}});
  }
  h_desc.resize(sizeof(Desc) * descs.size());
  std::memcpy(h_desc.data(), descs.data(), h_desc.size());
  if (cudaMemcpyAsync(d_desc, h_desc.data(), h_desc.size(), cudaMemcpyHostToDevice, sched)) return SIPG_ERR_CUDA;
  if (cudaMemcpyAsync(d_tiles, h_tiles.data(), sizeof(int2) * h_tiles.size(), cudaMemcpyHostToDevice, sched))
    return SIPG_ERR_CUDA;
  for (auto& gp : groups) {
    const int k = gp.first;
    const Tab& tab = by_k.at(k).front()->ctx->tabs[k + 1];
    cudaError_t e = std::is_same<TN, ff>::value
                        ? launch_apply_multi_ff(k + 1, 3, d_desc, d_tiles + gp.second.first, (int)gp.second.second,
                                                tab, sched)
                        : launch_apply_multi_f64(k + 1, 3, d_desc, d_tiles + gp.second.first,
                                                 (int)gp.second.second, tab, sched);
    if (e) return SIPG_ERR_CUDA;
  }
  return SIPG_OK;
}

// One CG iteration of every active request; the fine-level applies are batched.
int sipg_server::round() {
  // (1) each request's previous work is done before the batched apply reads p
  for (Request* r : active)
    if (cudaEventRecord(r->ev_ready, r->ctx->st)) return SIPG_ERR_CUDA;
  for (Request* r : active)
    if (cudaStreamWaitEvent(sched, r->ev_ready, 0)) return SIPG_ERR_CUDA;
  // (2) q_i = A_i p_i: one persistent launch per degree present
  std::map<int, std::vector<Request*>> by_k;
  for (Request* r : active) by_k[r->spec.k_u].push_back(r);
  const int brc = opts.krylov_arith == SIPG_F64_FF ? batched_apply<ff>(by_k) : batched_apply<double>(by_k);
  if (brc) return brc;
  if (cudaEventRecord(ev_applied, sched)) return SIPG_ERR_CUDA;
  // (copies from pageable host memory return once the source is consumed, so
  // the host tables may be rebuilt next round without waiting here)
  // (3) per request: alpha, x, r, ||r||, V-cycle, beta, p on its own stream
  for (Request* r : active) {
    sipg_ctx* ctx = r->ctx;
    cudaStream_t st = ctx->st;
    Hier& H = ctx->hier[SIPG_OP_VISCOUS];
    double *rr = H.cg[0], *z = H.cg[1], *p = H.cg[2], *q = H.cg[3];
    const int64_t n = r->n;
    if (cudaStreamWaitEvent(st, ev_applied, 0)) return SIPG_ERR_CUDA;
    if (launch_dot(n, p, q, ctx->partials, r->sc + 1, st)) return SIPG_ERR_CUDA;
    cg_check<<<1, 1, 0, st>>>(r->sc);
    cg_step_x_r<<<vec_blocks(n), 256, 0, st>>>(n, r->sc, p, q, r->x, rr);
    if (launch_dot(n, rr, rr, ctx->partials, r->sc + 2, st)) return SIPG_ERR_CUDA;
    if (cudaMemcpyAsync(r->hsc, r->sc + 2, sizeof(double), cudaMemcpyDeviceToHost, st)) return SIPG_ERR_CUDA;
    if (cudaMemcpyAsync(r->hsc + 1, r->sc + 5, sizeof(double), cudaMemcpyDeviceToHost, st)) return SIPG_ERR_CUDA;
    if (cudaEventRecord(r->ev_rr, st)) return SIPG_ERR_CUDA;
    int rc = ctx->precondition(SIPG_OP_VISCOUS, SIPG_PRECOND_MG, rr, z, 0.0);
    if (rc) return rc;
    if (launch_dot(n, rr, z, ctx->partials, r->sc + 3, st)) return SIPG_ERR_CUDA;
    cg_step_p<<<vec_blocks(n), 256, 0, st>>>(n, r->sc, z, p);
    cg_rotate<<<1, 1, 0, st>>>(r->sc);
    if (cudaGetLastError()) return SIPG_ERR_CUDA;
    r->iters++;
  }
  // (4) convergence from this round's residual norms (V-cycles keep running)
  std::vector<Request*> still;
  for (Request* r : active) {
    if (cudaEventSynchronize(r->ev_rr)) return SIPG_ERR_CUDA;
    const double res = std::sqrt(std::max(r->hsc[0], 0.0));
    const bool broke = r->hsc[1] != 0.0 || !std::isfinite(res);
    const bool conv = res <= r->spec.rtol * r->bnorm;
    if (conv && !broke) {
      bool restarted = false;
      int rc = confirm_or_restart(r, &restarted);
      if (rc) return rc;
      if (restarted) {
        still.push_back(r);
        continue;
      }
    }
    if (conv || broke || r->iters >= r->spec.maxit) {
      r->result.status = conv ? SIPG_OK : (broke ? SIPG_ERR_BREAKDOWN : SIPG_ERR_MAXIT);
      int rc = finish(r);
      if (rc) return rc;
    } else {
      still.push_back(r);
    }
  }
  active.swap(still);
  return SIPG_OK;
}

// The recursive residual met the tolerance: confirm it with the true residual
// b - A x. On large, high-contrast systems rounding in the recursion can leave the
// true residual a few times above the recursive one; then CG restarts from the
// true residual (r = b - A x, z = M r, p = z), at most kMaxReplacements times and
// within maxit, instead of returning a solution above the tolerance.
constexpr int kMaxReplacements = 3;
int sipg_server::confirm_or_restart(Request* r, bool* restarted) {
  *restarted = false;
  if (r->replacements >= kMaxReplacements || r->iters >= r->spec.maxit) return SIPG_OK;
  sipg_ctx* ctx = r->ctx;
  cudaStream_t st = ctx->st;
  Hier& H = ctx->hier[SIPG_OP_VISCOUS];
  double *rr = H.cg[0], *z = H.cg[1], *p = H.cg[2], *t = H.cg[3];
  const int64_t n = r->n;
  int rc = ctx->krylov_apply(SIPG_OP_VISCOUS, r->x, t, 0.0);
  if (rc) return rc;
  if (launch_sub<double>(n, r->b, t, rr, st)) return SIPG_ERR_CUDA;
  double rr2 = 0.0;
  if ((rc = ctx->dot(n, rr, rr, &rr2))) return rc;
  if (std::sqrt(rr2) <= r->spec.rtol * r->bnorm) return SIPG_OK;
  rc = ctx->precondition(SIPG_OP_VISCOUS, SIPG_PRECOND_MG, rr, z, 0.0);
  if (rc) return rc;
  if (cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st)) return SIPG_ERR_CUDA;
  if (launch_dot(n, rr, z, ctx->partials, r->sc + 0, st)) return SIPG_ERR_CUDA;
  r->replacements++;
  *restarted = true;
  return SIPG_OK;
}

// Final true residual, error against u*, optional copy of x; frees the slot.
int sipg_server::finish(Request* r) {
  sipg_ctx* ctx = r->ctx;
  cudaStream_t st = ctx->st;
  Hier& H = ctx->hier[SIPG_OP_VISCOUS];
  double *t = H.cg[3], *rr = H.cg[0];
  const int64_t n = r->n;
  int rc = ctx->krylov_apply(SIPG_OP_VISCOUS, r->x, t, 0.0);
  if (rc) return rc;
  if (launch_sub<double>(n, r->b, t, rr, st)) return SIPG_ERR_CUDA;
  double rr2 = 0.0, ee = 0.0, uu = 0.0;
  if ((rc = ctx->dot(n, rr, rr, &rr2))) return rc;
  const bool manufactured = r->spec.rhs == SIPG_RHS_MANUFACTURED;
  if (manufactured) {
    if (launch_sub<double>(n, r->x, r->ustar, t, st)) return SIPG_ERR_CUDA;
    if ((rc = ctx->dot(n, t, t, &ee))) return rc;
    if ((rc = ctx->dot(n, r->ustar, r->ustar, &uu))) return rc;
  }
  if (r->keep_solution) {
    r->solution.resize(n);
    if (cudaMemcpyAsync(r->solution.data(), r->x, sizeof(double) * n, cudaMemcpyDeviceToHost, st)) return SIPG_ERR_CUDA;
    if (cudaStreamSynchronize(st)) return SIPG_ERR_CUDA;
  }
  r->t_done = Clock::now();
  r->result.iterations = r->iters;
  r->result.rel_residual = r->bnorm > 0 ? std::sqrt(rr2) / r->bnorm : std::sqrt(rr2);
  r->result.err_vs_ustar = manufactured ? (uu > 0 ? std::sqrt(ee / uu) : 0.0) : std::nan("");
  r->result.n_dofs = n;
  r->result.queue_s = std::chrono::duration<double>(r->t_admit - r->t_submit).count();
  r->result.latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  r->result.solve_s = std::chrono::duration<double>(r->t_done - r->t_admit).count();
  for (ContextEntry& c : pool)
    if (c.ctx == ctx) c.busy = false;
  r->ctx = nullptr;
  r->done = true;
  return SIPG_OK;
}

void sipg_server::run() {
  if (cudaSetDevice(device) != cudaSuccess) {
    std::lock_guard<std::mutex> lk(mu);
    set_error("server worker: cudaSetDevice failed");
    cv_done.notify_all();
    return;
  }
  while (true) {
    // admission (between rounds)
    std::vector<std::unique_ptr<Request>> admitted;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] { return stop || !queue.empty() || !active.empty(); });
      if (stop && queue.empty() && active.empty()) break;
      while (!queue.empty() && (int)active.size() + (int)admitted.size() < opts.max_slots) {
        std::unique_ptr<Request>& rq = queue.front();
        if (!admit_one(rq)) break;  // memory busy: retry after the next round
        admitted.push_back(std::move(rq));
        queue.pop_front();
      }
    }
    for (auto& up : admitted) {
      Request* r = up.get();
      if (!r->done) {
        int rc = start_request(r);
        if (rc) {
          r->result.status = rc;
          r->done = true;
          for (ContextEntry& c : pool)
            if (c.ctx == r->ctx) c.busy = false;
        } else {
          active.push_back(r);
        }
      }
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      for (auto& up : admitted) {
        const uint64_t id = up->id;
        if (up->done) --pending;
        finished[id] = std::move(up);
      }
    }
    if (active.empty()) {
      cv_done.notify_all();
      continue;
    }
    std::vector<Request*> before = active;
    int rc = round();
    std::lock_guard<std::mutex> lk(mu);
    if (rc) {
      set_error("server round failed with status " + std::to_string(rc));
      for (Request* r : before) {
        r->result.status = rc;
        r->done = true;
      }
      active.clear();
    }
    for (Request* r : before)
      if (r->done) --pending;
    cv_done.notify_all();
  }
}

// ---------------------------------------------------------------- C ABI
extern "C" int sipg_server_create(const sipg_server_opts* o, sipg_server** out) {
  if (!o || !out || o->max_slots <= 0 || o->hbm_budget_bytes == 0) return SIPG_ERR_INVALID;
  if (o->mg_precision != SIPG_F32 && o->mg_precision != SIPG_F64) return SIPG_ERR_INVALID;
  if (o->krylov_arith != SIPG_F64 && o->krylov_arith != SIPG_F64_FF) return SIPG_ERR_INVALID;
  auto* s = new sipg_server();
  s->opts = *o;
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->sched, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_applied, cudaEventDisableTiming) != cudaSuccess) {
    delete s;
    return SIPG_ERR_CUDA;
  }
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return SIPG_OK;
}

extern "C" int sipg_server_submit(sipg_server* s, const sipg_request* req, uint64_t* id) {
  if (!s || !req || !id || !req->rheology) return SIPG_ERR_INVALID;
  const sipg_rheology& rh = *req->rheology;
  if (req->n_cells <= 0 || req->n_cells > 1024 || req->k_u < 2 || req->k_u > 5 || !(req->rtol > 0) ||
      req->maxit <= 0)
    return SIPG_ERR_INVALID;
  if (rh.law != SIPG_LAW_CONSTANT && rh.law != SIPG_LAW_ANALYTIC && rh.law != SIPG_LAW_SINKER)
    return SIPG_ERR_INVALID;  // served solves are linear: no velocity-dependent law
  if (rh.law == SIPG_LAW_SINKER &&
      (rh.n_spheres < 0 || rh.n_spheres > 64 || (rh.n_spheres > 0 && !rh.centers) || !(rh.nu_max > 0) ||
       !(rh.nu_matrix > 0) || !(rh.radius >= 0)))
    return SIPG_ERR_INVALID;
  if (rh.law == SIPG_LAW_CONSTANT && !(rh.nu > 0)) return SIPG_ERR_INVALID;
  if (req->rhs < SIPG_RHS_MANUFACTURED || req->rhs > SIPG_RHS_DEVICE) return SIPG_ERR_INVALID;
  if ((req->rhs == SIPG_RHS_HOST || req->rhs == SIPG_RHS_DEVICE) && !req->b) return SIPG_ERR_INVALID;
  auto r = std::make_unique<Request>();
  r->spec = *req;
  r->spec.rheology = nullptr;
  r->rh = rh;
  if (rh.law == SIPG_LAW_SINKER) r->centers.assign(rh.centers, rh.centers + 3 * rh.n_spheres);
  r->rh.centers = nullptr;
  if (req->rhs == SIPG_RHS_HOST) {
    const int64_t nk = req->k_u + 1;
    const int64_t n = (int64_t)req->n_cells * req->n_cells * req->n_cells * 3 * nk * nk * nk;
    r->b_host.assign(req->b, req->b + n);
    r->spec.b = nullptr;
  }
  r->keep_solution = req->keep_solution != 0;
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->failed) return SIPG_ERR_STATE;
  r->id = s->next_id++;
  *id = r->id;
  s->queue.push_back(std::move(r));
  ++s->pending;
  s->cv.notify_all();
  return SIPG_OK;
}

extern "C" int sipg_server_poll(sipg_server* s, uint64_t id, sipg_result* res, double* x_host) {
  if (!s || !res) return SIPG_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->finished.find(id);
  if (it == s->finished.end() || !it->second->done) {
    for (const auto& q : s->queue)
      if (q->id == id) return SIPG_PENDING;
    if (it != s->finished.end()) return SIPG_PENDING;
    return id < s->next_id ? SIPG_PENDING : SIPG_ERR_INVALID;
  }
  *res = it->second->result;
  if (x_host && !it->second->solution.empty())
    std::memcpy(x_host, it->second->solution.data(), sizeof(double) * it->second->solution.size());
  return SIPG_OK;
}

extern "C" int sipg_server_drain(sipg_server* s, double timeout_s) {
  if (!s) return SIPG_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9);
  while (s->pending > 0 && !s->failed) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && s->pending > 0) return SIPG_ERR_TIMEOUT;
  }
  return s->failed ? SIPG_ERR_STATE : SIPG_OK;
}

extern "C" const char* sipg_server_last_error(const sipg_server* s) { return s ? s->err.c_str() : "null server"; }

extern "C" int sipg_server_destroy(sipg_server* s) {
  if (!s) return SIPG_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (ContextEntry& c : s->pool) s->release_entry(c);
  cudaFree(s->d_desc);
  cudaFree(s->d_tiles);
  cudaEventDestroy(s->ev_applied);
  cudaStreamDestroy(s->sched);
  delete s;
  return SIPG_OK;
}
