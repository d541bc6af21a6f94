// Register-tiled FP32 operator kernel (operator_tpc.cuh): instantiations and
// launch for n = 2, 3, 4.
#include "kernels.cuh"
#include "operator_tpc.cuh"

namespace sipg {

namespace {

TpcTab make_tpc_tab(const Tab& t) {
  TpcTab c{};
  for (int i = 0; i < kMaxN * kMaxN; ++i) {
    c.S[i] = (float)t.S[i];
    c.Dg[i] = (float)t.Dg[i];
  }
  for (int i = 0; i < kMaxN; ++i) {
    c.dS0[i] = (float)t.dS0[i];
    c.dS1[i] = (float)t.dS1[i];
    c.gw[i] = (float)t.gw[i];
  }
  return c;
}

template <int N, int NC, bool TOPO>
cudaError_t launch_tpc_g(const LevelGeom& g, const Tab& tab, const float* x, float* y, const float* nu_cell,
                         const float* nu_face, float mass, int nbatch, cudaStream_t st) {
  constexpr int CW = TpcCfg<NC>::CW;
  const size_t smem = sizeof(float) * tpc_smem_floats<N, NC>();
  static bool attr_set = false;  // per instantiation, per process (single device)
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(apply_tpc_kernel<N, NC, TOPO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int grid = (g.ncells + CW - 1) / CW;
  if (grid == 0 || nbatch == 0) return cudaSuccess;
  const int64_t stride = (int64_t)g.ncells * NC * N * N * N;
  apply_tpc_kernel<N, NC, TOPO><<<dim3(grid, nbatch), 32, smem, st>>>(
      g, make_tpc_tab(tab), level_consts<float>(g, N, mass), x, y, nu_cell, nu_face, stride);
  return cudaGetLastError();
}

template <int N, int NC>
cudaError_t launch_tpc_n(const LevelGeom& g, const Tab& tab, const float* x, float* y, const float* nu_cell,
                         const float* nu_face, float mass, int nbatch, cudaStream_t st) {
  return g.nbr ? launch_tpc_g<N, NC, true>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st)
               : launch_tpc_g<N, NC, false>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st);
}

}  // namespace

bool tpc_supported(int n) { return n >= 2 && n <= 4; }

cudaError_t launch_apply_tpc(int n, int ncomp, const LevelGeom& g, const Tab& tab, const float* x, float* y,
                             const float* nu_cell, const float* nu_face, float mass, int nbatch, cudaStream_t st) {
  switch (n) {
    case 2:
      return ncomp == 3 ? launch_tpc_n<2, 3>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st)
                        : launch_tpc_n<2, 1>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st);
    case 3:
      return ncomp == 3 ? launch_tpc_n<3, 3>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st)
                        : launch_tpc_n<3, 1>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st);
    case 4:
      return ncomp == 3 ? launch_tpc_n<4, 3>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st)
                        : launch_tpc_n<4, 1>(g, tab, x, y, nu_cell, nu_face, mass, nbatch, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace sipg
