// Continuous ("cph") multigrid levels (Sec. 5.4: the hp-multigrid first
// converts the DG space to the continuous space of the same degree, then lowers
// the degree, then coarsens the mesh). On the box with structured cells and
// Gauss-Lobatto nodes a continuous vector holds one value per node of the
// global (nx k + 1) x (ny k + 1) x (nz k + 1) grid and component
// (component-major). The level operator is P^T A_DG P, evaluated as gather ->
// DG operator kernel -> sum over the copies; these kernels are the maps:
//   gather      P:   DG coefficient of (cell, comp, local node) = global value
//   scatter_sum P^T: global value = sum of the DG coefficients of its copies
//   pick        R:   global value = copy in the lowest-index cell holding it
//   pick_t      R^T: that copy gets the global value, the other copies 0
// One thread per output entry; deterministic (no atomics). blockIdx.y selects
// one vector of a batch (the coarse-level assembly).
#include "kernels.cuh"

namespace sipg {
namespace {

constexpr int kCphThreads = 256;

__device__ __forceinline__ void lowest_copy(int g, int k, int& cell, int& local) {
  if (g > 0 && g % k == 0) {
    cell = g / k - 1;
    local = k;
  } else {
    cell = g / k;
    local = g % k;
  }
}

template <typename T>
__global__ void gather_kernel(CgGrid cg, const T* __restrict__ x, T* __restrict__ y, int64_t ncg, int64_t ndg) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ndg) return;
  x += (int64_t)blockIdx.y * ncg;
  y += (int64_t)blockIdx.y * ndg;
  const int n = cg.k + 1, n3 = n * n * n;
  const int64_t ec = t / n3;
  const int loc = (int)(t - ec * n3);
  const int c = (int)(ec % cg.ncomp);
  const int64_t e = ec / cg.ncomp;
  const int i = (int)(e % cg.nx), j = (int)((e / cg.nx) % cg.ny), l = (int)(e / ((int64_t)cg.nx * cg.ny));
  const int ix = loc % n, iy = (loc / n) % n, iz = loc / (n * n);
  const int64_t gidx = ((int64_t)(l * cg.k + iz) * cg.Gy + (j * cg.k + iy)) * cg.Gx + (i * cg.k + ix);
  y[t] = x[(int64_t)c * cg.Gx * cg.Gy * cg.Gz + gidx];
}

template <typename T>
__global__ void scatter_sum_kernel(CgGrid cg, const T* __restrict__ x, T* __restrict__ y, int64_t ncg, int64_t ndg) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ncg) return;
  x += (int64_t)blockIdx.y * ndg;
  y += (int64_t)blockIdx.y * ncg;
  const int64_t Ng = (int64_t)cg.Gx * cg.Gy * cg.Gz;
  const int c = (int)(t / Ng);
  const int64_t gi = t - c * Ng;
  const int g[3] = {(int)(gi % cg.Gx), (int)((gi / cg.Gx) % cg.Gy), (int)(gi / ((int64_t)cg.Gx * cg.Gy))};
  const int nc[3] = {cg.nx, cg.ny, cg.nz};
  const int n = cg.k + 1;
  int cells[3][2], locs[3][2], cnt[3];
  for (int d = 0; d < 3; ++d) {
    cnt[d] = 0;
    const int q = g[d] / cg.k, r = g[d] % cg.k;
    if (q < nc[d]) {
      cells[d][cnt[d]] = q;
      locs[d][cnt[d]] = r;
      ++cnt[d];
    }
    if (r == 0 && q > 0) {
      cells[d][cnt[d]] = q - 1;
      locs[d][cnt[d]] = cg.k;
      ++cnt[d];
    }
  }
  T acc = T(0);
  for (int a = 0; a < cnt[0]; ++a)
    for (int b = 0; b < cnt[1]; ++b)
      for (int z = 0; z < cnt[2]; ++z) {
        const int64_t e = ((int64_t)cells[2][z] * cg.ny + cells[1][b]) * cg.nx + cells[0][a];
        const int loc = (locs[2][z] * n + locs[1][b]) * n + locs[0][a];
        acc += x[(e * cg.ncomp + c) * n * n * n + loc];
      }
  y[t] = acc;
}

template <typename T>
__global__ void pick_kernel(CgGrid cg, const T* __restrict__ x, T* __restrict__ y, int64_t ncg) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ncg) return;
  const int64_t Ng = (int64_t)cg.Gx * cg.Gy * cg.Gz;
  const int c = (int)(t / Ng);
  const int64_t gi = t - c * Ng;
  const int g[3] = {(int)(gi % cg.Gx), (int)((gi / cg.Gx) % cg.Gy), (int)(gi / ((int64_t)cg.Gx * cg.Gy))};
  int cell[3], loc[3];
  for (int d = 0; d < 3; ++d) lowest_copy(g[d], cg.k, cell[d], loc[d]);
  const int n = cg.k + 1;
  const int64_t e = ((int64_t)cell[2] * cg.ny + cell[1]) * cg.nx + cell[0];
  y[t] = x[(e * cg.ncomp + c) * n * n * n + (loc[2] * n + loc[1]) * n + loc[0]];
}

template <typename T>
__global__ void pick_t_kernel(CgGrid cg, const T* __restrict__ x, T* __restrict__ y, int64_t ndg) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ndg) return;
  const int n = cg.k + 1, n3 = n * n * n;
  const int64_t ec = t / n3;
  const int loc = (int)(t - ec * n3);
  const int c = (int)(ec % cg.ncomp);
  const int64_t e = ec / cg.ncomp;
  const int cell[3] = {(int)(e % cg.nx), (int)((e / cg.nx) % cg.ny), (int)(e / ((int64_t)cg.nx * cg.ny))};
  const int li[3] = {loc % n, (loc / n) % n, loc / (n * n)};
  // the lowest-index copy: no direction in which the node is the first node of a cell > 0
  bool lowest = true;
  for (int d = 0; d < 3; ++d) lowest = lowest && !(li[d] == 0 && cell[d] > 0);
  if (!lowest) {
    y[t] = T(0);
    return;
  }
  const int64_t gidx = ((int64_t)(cell[2] * cg.k + li[2]) * cg.Gy + (cell[1] * cg.k + li[1])) * cg.Gx +
                       (cell[0] * cg.k + li[0]);
  y[t] = x[(int64_t)c * cg.Gx * cg.Gy * cg.Gz + gidx];
}

}  // namespace

template <typename T>
cudaError_t launch_cg_map(int kind, const CgGrid& cg, const T* x, T* y, int nbatch, cudaStream_t st) {
  const int64_t ncg = (int64_t)cg.ncomp * cg.Gx * cg.Gy * cg.Gz;
  const int64_t ndg = (int64_t)cg.nx * cg.ny * cg.nz * cg.ncomp * (cg.k + 1) * (cg.k + 1) * (cg.k + 1);
  if (nbatch <= 0) return cudaSuccess;
  switch (kind) {
    case CG_GATHER:
      gather_kernel<T><<<dim3((unsigned)((ndg + kCphThreads - 1) / kCphThreads), nbatch), kCphThreads, 0, st>>>(
          cg, x, y, ncg, ndg);
      break;
    case CG_SCATTER_SUM:
      scatter_sum_kernel<T><<<dim3((unsigned)((ncg + kCphThreads - 1) / kCphThreads), nbatch), kCphThreads, 0, st>>>(
          cg, x, y, ncg, ndg);
      break;
    case CG_PICK:
      if (nbatch != 1) return cudaErrorInvalidValue;
      pick_kernel<T><<<(unsigned)((ncg + kCphThreads - 1) / kCphThreads), kCphThreads, 0, st>>>(cg, x, y, ncg);
      break;
    case CG_PICK_T:
      if (nbatch != 1) return cudaErrorInvalidValue;
      pick_t_kernel<T><<<(unsigned)((ndg + kCphThreads - 1) / kCphThreads), kCphThreads, 0, st>>>(cg, x, y, ndg);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t launch_cg_map<float>(int, const CgGrid&, const float*, float*, int, cudaStream_t);
template cudaError_t launch_cg_map<double>(int, const CgGrid&, const double*, double*, int, cudaStream_t);

}  // namespace sipg
