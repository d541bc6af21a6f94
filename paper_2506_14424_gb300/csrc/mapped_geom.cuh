// Geometry of trilinear (non-affine) hexahedra for the kernels of mapped.cu and
// mapped_split.cu: cell vertices, the Jacobian of the trilinear map and its
// inverse at a reference point, and the face evaluation / its transpose of a
// nodal field (values and reference derivatives at the face Gauss points).
// Device code only; one CTA per cell (split.cu style, shared-memory tensors).
#pragma once
#include "sweeps.cuh"

namespace sipg {
namespace mgeo {
using namespace sweeps;

template <typename R>
__device__ __forceinline__ void load_cell_vertices(const LevelGeom& g, const double* __restrict__ verts, int e,
                                                   R (*X)[3]) {
  int ijk[3];
  cell_ijk(g, e, ijk);
  const int i = ijk[0], j = ijk[1], k = ijk[2];
  for (int t = threadIdx.x; t < 24; t += blockDim.x) {
    const int v = t / 3, c = t % 3;
    const int a = v & 1, b = (v >> 1) & 1, cc = (v >> 2) & 1;
    const size_t idx = ((size_t)(k + cc) * (g.ny + 1) + (j + b)) * (g.nx + 1) + (i + a);
    X[v][c] = (R)verts[idx * 3 + c];
  }
}

// J[k][l] = d x_k / d xi_l of the trilinear map at xi; also x if wanted
template <typename R>
__device__ __forceinline__ void trilinear_jac(const R (*X)[3], R x0, R x1, R x2, R J[3][3], R* pos = nullptr) {
  for (int k = 0; k < 3; ++k) {
    J[k][0] = J[k][1] = J[k][2] = R(0);
    if (pos) pos[k] = R(0);
  }
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const int a = v & 1, b = (v >> 1) & 1, c = (v >> 2) & 1;
    const R fx = a ? x0 : R(1) - x0, fy = b ? x1 : R(1) - x1, fz = c ? x2 : R(1) - x2;
    const R sx = a ? R(1) : R(-1), sy = b ? R(1) : R(-1), sz = c ? R(1) : R(-1);
    const R d0 = sx * fy * fz, d1 = fx * sy * fz, d2 = fx * fy * sz;
    for (int k = 0; k < 3; ++k) {
      J[k][0] += X[v][k] * d0;
      J[k][1] += X[v][k] * d1;
      J[k][2] += X[v][k] * d2;
      if (pos) pos[k] += X[v][k] * fx * fy * fz;
    }
  }
}

template <typename R>
__device__ __forceinline__ R inverse3(const R J[3][3], R Ji[3][3]) {
  const R c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const R c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const R c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const R det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  const R id = R(1) / det;
  Ji[0][0] = c00 * id;
  Ji[1][0] = c01 * id;
  Ji[2][0] = c02 * id;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  return det;
}

// node (layer along d, a along t1, b along t2) of an n^3 tensor
__device__ __forceinline__ int lnode(int d, int layer, int a, int b, int n) {
  int i[3];
  int t1, t2;
  face_dirs(d, &t1, &t2);
  i[d] = layer;
  i[t1] = a;
  i[t2] = b;
  return (i[2] * n + i[1]) * n + i[0];
}

// Values and reference derivatives at the face Gauss points of a nodal field U
// (n^3): out[0] values, out[1] d/dxi_d, out[2] d/dxi_t1, out[3] d/dxi_t2 (N^2
// each); scratch: 5 N^2.
template <int N, typename R>
__device__ void face_eval(const R* U, int d, int s, const STabSmT<R>& T, R* out, R* sc) {
  constexpr int N2 = N * N;
  R *L = sc, *D = sc + N2, *A = sc + 2 * N2, *B = sc + 3 * N2, *C = sc + 4 * N2;
  for (int p = threadIdx.x; p < N2; p += blockDim.x) {
    const int a = p % N, b = p / N;
    L[p] = U[lnode(d, s ? N - 1 : 0, a, b, N)];
    R acc = R(0);
#pragma unroll
    for (int i = 0; i < N; ++i) acc += T.dS[s][i] * U[lnode(d, i, a, b, N)];
    D[p] = acc;
  }
  __syncthreads();
  sweep<N, N, 1, 0, N, false>(T.S, N, L, A);
  sweep<N, N, 1, 0, N, false>(T.DS, N, L, B);
  sweep<N, N, 1, 0, N, false>(T.S, N, D, C);
  __syncthreads();
  sweep<N, N, 1, 1, N, false>(T.S, N, A, out);            // values
  sweep<N, N, 1, 1, N, false>(T.S, N, C, out + N2);       // d/dxi_d
  sweep<N, N, 1, 1, N, false>(T.S, N, B, out + 2 * N2);   // d/dxi_t1
  sweep<N, N, 1, 1, N, false>(T.DS, N, A, out + 3 * N2);  // d/dxi_t2
  __syncthreads();
}

// Transpose of face_eval: add to the nodal tensor Y the test-side contributions
// of coefficients cf[0] (value), cf[1] (d/dxi_d), cf[2] (d/dxi_t1), cf[3] (d/dxi_t2).
template <int N, typename R>
__device__ void face_eval_t(const R* cf, int d, int s, const STabSmT<R>& T, R* Y, R* sc) {
  constexpr int N2 = N * N, N3 = N2 * N;
  R *A = sc, *B = sc + N2, *C = sc + 2 * N2, *L = sc + 3 * N2, *D = sc + 4 * N2;
  sweep<N, N, 1, 1, N, true>(T.S, N, cf, A);
  sweep<N, N, 1, 1, N, true>(T.S, N, cf + N2, C);
  sweep<N, N, 1, 1, N, true>(T.S, N, cf + 2 * N2, B);
  __syncthreads();
  sweep<N, N, 1, 0, N, true>(T.S, N, A, L);   // value part
  sweep<N, N, 1, 0, N, true>(T.S, N, C, D);   // normal part
  __syncthreads();
  sweep<N, N, 1, 0, N, true>(T.DS, N, B, A);  // d/dxi_t1 part (A is free again)
  sweep<N, N, 1, 1, N, true>(T.DS, N, cf + 3 * N2, C);
  __syncthreads();
  for (int p = threadIdx.x; p < N2; p += blockDim.x) L[p] += A[p];
  sweep<N, N, 1, 0, N, true>(T.S, N, C, B);   // d/dxi_t2 part
  __syncthreads();
  for (int p = threadIdx.x; p < N2; p += blockDim.x) A[p] = L[p] + B[p];
  __syncthreads();
  // layer nodes: values and tangential parts; every node along the normal line: normal part
  for (int i = threadIdx.x; i < N3; i += blockDim.x) {
    const int idx[3] = {i % N, (i / N) % N, i / N2};
    int t1, t2;
    face_dirs(d, &t1, &t2);
    const int p = idx[t1] + N * idx[t2];
    R v = T.dS[s][idx[d]] * D[p];
    if (idx[d] == (s ? N - 1 : 0)) v += A[p];
    Y[i] += v;
  }
  __syncthreads();
}


// 1D matrices of the trilinear apply as a kernel parameter: in the line sweeps
// below every matrix index is a compile-time constant, so S, DS and Dg are
// constant-bank operands of the multiply-adds (no shared-memory loads of the
// matrices, one thread per line instead of one per output entry)
template <typename R>
struct MTab {
  R S[kMaxN * kMaxN], DS[kMaxN * kMaxN], Dg[kMaxN * kMaxN];
};
template <typename R>
inline MTab<R> make_mtab(const SplitTab& t) {
  MTab<R> m{};
  for (int i = 0; i < kMaxN * kMaxN; ++i) {
    m.S[i] = (R)t.S[i];
    m.DS[i] = (R)t.DS[i];
    m.Dg[i] = (R)t.Dg[i];
  }
  return m;
}

// out (+)= M along DIR on ntens consecutive N^3 tensors (x fastest), one thread
// per 1D line: its N inputs in registers, N outputs; M(o, j) = M[o N + j], or
// M[j N + o] if TR
template <int N, int DIR, bool TR, bool ACC, typename R>
__device__ __forceinline__ void lsweep(const R* M, const R* __restrict__ in, R* __restrict__ out, int ntens) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr int STR = DIR == 0 ? 1 : (DIR == 1 ? N : N2);
  for (int line = threadIdx.x; line < ntens * N2; line += blockDim.x) {
    const int t = line / N2, r = line - t * N2;
    const int off = t * N3 + (DIR == 0 ? r * N : (DIR == 1 ? (r % N) + (r / N) * N2 : r));
    R v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = in[off + j * STR];
#pragma unroll
    for (int o = 0; o < N; ++o) {
      R acc = R(0);
#pragma unroll
      for (int j = 0; j < N; ++j) acc += (TR ? M[j * N + o] : M[o * N + j]) * v[j];
      R* dst = out + off + o * STR;
      *dst = ACC ? *dst + acc : acc;
    }
  }
}

// the same on ntens consecutive N^2 face tensors (a fastest): DIR 0 along a, 1 along b
template <int N, int DIR, bool TR, typename R>
__device__ __forceinline__ void lsweep2(const R* M, const R* __restrict__ in, R* __restrict__ out, int ntens) {
  constexpr int N2 = N * N;
  constexpr int STR = DIR == 0 ? 1 : N;
  for (int line = threadIdx.x; line < ntens * N; line += blockDim.x) {
    const int t = line / N, r = line - t * N;
    const int off = t * N2 + (DIR == 0 ? r * N : r);
    R v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = in[off + j * STR];
#pragma unroll
    for (int o = 0; o < N; ++o) {
      R acc = R(0);
#pragma unroll
      for (int j = 0; j < N; ++j) acc += (TR ? M[j * N + o] : M[o * N + j]) * v[j];
      out[off + o * STR] = acc;
    }
  }
}

// Line sweeps (one thread per line, matrices in the kernel parameter) or entry
// sweeps (one thread per output entry, matrices in shared memory): lines of an
// even degree count N >= 4 are 4-way bank-conflicted (stride N), so they keep the
// entry form. Measured at 32^3, 5 % jitter (FP32 level applies): n = 3 viscous
// 0.49 -> 0.39 ms, n = 3 pressure 0.22 -> 0.21 ms, n = 2 0.143 -> 0.136 ms with
// lines; n = 4 0.83 -> 1.22 ms (FP32) and 3.9 -> 5.0 ms (FP64) with lines.
template <int N>
__host__ __device__ constexpr bool mapped_line_sweeps() { return N == 2 || N % 2 == 1; }

// face_eval on ntens tensors at once: src(b, i) is node i of tensor b (shared or
// global memory); out: ntens x 4 N^2 ([b][slot][p]); sc: 6 ntens N^2 scratch
template <int N, typename R, typename Src>
__device__ __forceinline__ void face_evalb(Src src, int d, int s, const STabSmT<R>& T, const MTab<R>& mt, R* out,
                                           R* sc, int ntens) {
  constexpr int N2 = N * N;
  const int M = ntens * N2;
  R *L = sc, *D = sc + M, *A = sc + 2 * M, *B = sc + 3 * M, *C = sc + 4 * M, *E = sc + 5 * M;
  for (int t = threadIdx.x; t < M; t += blockDim.x) {
    const int b = t / N2, p = t - b * N2;
    const int a = p % N, c = p / N;
    L[t] = src(b, lnode(d, s ? N - 1 : 0, a, c, N));
    R acc = R(0);
#pragma unroll
    for (int i = 0; i < N; ++i) acc += T.dS[s][i] * src(b, lnode(d, i, a, c, N));
    D[t] = acc;
  }
  __syncthreads();
  if constexpr (mapped_line_sweeps<N>()) {
    // along a: A = S L, B = DS L, C = S D
    lsweep2<N, 0, false>(mt.S, L, A, ntens);
    lsweep2<N, 0, false>(mt.DS, L, B, ntens);
    lsweep2<N, 0, false>(mt.S, D, C, ntens);
    __syncthreads();
    // along b: values E = S A, d/dxi_d L = S C, d/dxi_t1 D = S B (inputs and outputs disjoint)
    lsweep2<N, 1, false>(mt.S, A, E, ntens);
    lsweep2<N, 1, false>(mt.S, C, L, ntens);
    lsweep2<N, 1, false>(mt.S, B, D, ntens);
    __syncthreads();
    lsweep2<N, 1, false>(mt.DS, A, C, ntens);  // d/dxi_t2 = DS_b A
    __syncthreads();
  } else {
    sweepb<N, N, 1, 0, N, false>(T.S, N, L, A, ntens);
    sweepb<N, N, 1, 0, N, false>(T.DS, N, L, B, ntens);
    sweepb<N, N, 1, 0, N, false>(T.S, N, D, C, ntens);
    __syncthreads();
    sweepb<N, N, 1, 1, N, false>(T.S, N, A, E, ntens);
    sweepb<N, N, 1, 1, N, false>(T.S, N, C, L, ntens);
    sweepb<N, N, 1, 1, N, false>(T.S, N, B, D, ntens);
    __syncthreads();
    sweepb<N, N, 1, 1, N, false>(T.DS, N, A, C, ntens);
    __syncthreads();
  }
  for (int t = threadIdx.x; t < M; t += blockDim.x) {
    const int b = t / N2, p = t - b * N2;
    R* o = out + b * 4 * N2 + p;
    o[0] = E[t];
    o[N2] = L[t];
    o[2 * N2] = D[t];
    o[3 * N2] = C[t];
  }
  __syncthreads();
}

// face_eval_t on ntens tensors: coefficients cf (ntens x 4 N^2, [b][slot][p]) added
// to Y (ntens x N^3); sc: 8 ntens N^2 scratch
template <int N, typename R>
__device__ __forceinline__ void face_eval_tb(const R* cf, int d, int s, const STabSmT<R>& T, const MTab<R>& mt, R* Y,
                                             R* sc, int ntens) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const int M = ntens * N2;
  R *V0 = sc, *V1 = sc + M, *V2 = sc + 2 * M, *V3 = sc + 3 * M;
  R *Pv = sc + 4 * M, *Pn = sc + 5 * M, *P1 = sc + 6 * M, *P2 = sc + 7 * M;
  for (int t = threadIdx.x; t < M; t += blockDim.x) {
    const int b = t / N2, p = t - b * N2;
    const R* c = cf + b * 4 * N2 + p;
    V0[t] = c[0];
    V1[t] = c[N2];
    V2[t] = c[2 * N2];
    V3[t] = c[3 * N2];
  }
  __syncthreads();
  // along b (transposed): value S^T, normal S^T, t1 S^T, t2 DS^T
  if constexpr (mapped_line_sweeps<N>()) {
    lsweep2<N, 1, true>(mt.S, V0, Pv, ntens);
    lsweep2<N, 1, true>(mt.S, V1, Pn, ntens);
    lsweep2<N, 1, true>(mt.S, V2, P1, ntens);
    lsweep2<N, 1, true>(mt.DS, V3, P2, ntens);
  } else {
    sweepb<N, N, 1, 1, N, true>(T.S, N, V0, Pv, ntens);
    sweepb<N, N, 1, 1, N, true>(T.S, N, V1, Pn, ntens);
    sweepb<N, N, 1, 1, N, true>(T.S, N, V2, P1, ntens);
    sweepb<N, N, 1, 1, N, true>(T.DS, N, V3, P2, ntens);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < M; t += blockDim.x) Pv[t] += P2[t];  // value and t2 parts share S_a^T
  __syncthreads();
  // along a (transposed): (value + t2) S^T, normal S^T, t1 DS^T
  if constexpr (mapped_line_sweeps<N>()) {
    lsweep2<N, 0, true>(mt.S, Pv, V0, ntens);
    lsweep2<N, 0, true>(mt.S, Pn, V1, ntens);
    lsweep2<N, 0, true>(mt.DS, P1, V2, ntens);
  } else {
    sweepb<N, N, 1, 0, N, true>(T.S, N, Pv, V0, ntens);
    sweepb<N, N, 1, 0, N, true>(T.S, N, Pn, V1, ntens);
    sweepb<N, N, 1, 0, N, true>(T.DS, N, P1, V2, ntens);
  }
  __syncthreads();
  // layer nodes: values and tangential parts; every node along the normal line: normal part
  int t1, t2;
  face_dirs(d, &t1, &t2);
  for (int i = threadIdx.x; i < ntens * N3; i += blockDim.x) {
    const int b = i / N3, r = i - b * N3;
    const int idx[3] = {r % N, (r / N) % N, r / N2};
    const int p = b * N2 + idx[t1] + N * idx[t2];
    R v = T.dS[s][idx[d]] * V1[p];
    if (idx[d] == (s ? N - 1 : 0)) v += V0[p] + V2[p];
    Y[i] += v;
  }
  __syncthreads();
}

}  // namespace mgeo
}  // namespace sipg
