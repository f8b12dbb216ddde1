// Macro-scale kernels: Fbar at the macro quadrature points and the HMM assembly of the
// macro residual and tangent on a structured Q1 (2D) / Hex8 (3D) mesh of [0,1]^d.
//
// Paper Sec. 3.1-3.2: Fbar = I + Grad u^H at x_{K_delta_l} (the gradient of the
// linearised macro field, Eq. linearization-uH); f_I = sum_qp omega Pbar Grad N_I, which is
// int B_I^T S^H with S^H = <F>^-1 <P> (Eq. f_I^int, macro-mean-stress); and
// K_IJ = sum_qp omega Grad N_I . Abar . Grad N_J, the RVE-averaged bilinear form of
// Eq. ModifiedBilinearForm-3 assembled as in Eq. Assem_k_T_IK_mac.
//
// The assembly is a graph-coloured scatter: elements are split into 2^d colours by the
// parity of their grid coordinates, so no two elements of one colour share a node and each
// colour's launch adds into f and the CSR values without atomics (deterministic sums).
// One thread computes one d x d block (I, J) of one element.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rve_args.h"

namespace fehmm {
namespace {

__device__ __forceinline__ double gauss01(int g) {
  return g == 0 ? 0.21132486540518711775 : 0.78867513459481288225;
}
__device__ __forceinline__ int cx(int a) { return ((a & 3) == 1 || (a & 3) == 2) ? 1 : 0; }
__device__ __forceinline__ int cy(int a) { return (a & 3) >= 2 ? 1 : 0; }
__device__ __forceinline__ int cz(int a) { return a >= 4 ? 1 : 0; }

// physical gradient of corner a's shape function at Gauss point g
template <int D>
__device__ __forceinline__ void grad_N(int a, int g, const MacroArgs& m, double (&gr)[3]) {
  const double xi[3] = {gauss01(g & 1), gauss01((g >> 1) & 1), D == 3 ? gauss01((g >> 2) & 1) : 0.0};
  const int of[3] = {cx(a), cy(a), cz(a)};
  double phi[3], dphi[3];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    phi[k] = of[k] ? xi[k] : 1.0 - xi[k];
    dphi[k] = of[k] ? 1.0 : -1.0;
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double v = dphi[k] / m.h[k];
#pragma unroll
    for (int l = 0; l < D; ++l)
      if (l != k) v *= phi[l];
    gr[k] = v;
  }
}

template <int D>
__device__ __forceinline__ int corner_node(int e, int a, const MacroArgs& m) {
  const int ex = e % m.nel[0], ey = (e / m.nel[0]) % m.nel[1], ez = D == 3 ? e / (m.nel[0] * m.nel[1]) : 0;
  const int nx1 = m.nel[0] + 1, ny1 = m.nel[1] + 1;
  return (ex + cx(a)) + nx1 * (ey + cy(a)) + (D == 3 ? nx1 * ny1 * (ez + cz(a)) : 0);
}

template <int D>
__global__ void macro_qp_F_kernel(const MacroArgs m) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m.n_qp) return;
  const int e = q / m.nq, g = q % m.nq;
  double F[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int J = 0; J < D; ++J) F[i][J] = (i == J) ? 1.0 : 0.0;
#pragma unroll
  for (int a = 0; a < (1 << D); ++a) {
    double gr[3];
    grad_N<D>(a, g, m, gr);
    const int node = corner_node<D>(e, a, m);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const double ui = m.u[(size_t)node * D + i];
#pragma unroll
      for (int J = 0; J < D; ++J) F[i][J] += ui * gr[J];
    }
  }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int J = 0; J < D; ++J) m.F[(size_t)q * D * D + i * D + J] = F[i][J];
}

template <int D>
__global__ void macro_assemble_kernel(const MacroArgs m, int color) {
  constexpr int NEN = 1 << D, NQ = 1 << D;
  const int c0 = color & 1, c1 = (color >> 1) & 1, c2 = (color >> 2) & 1;
  const int n0 = (m.nel[0] - c0 + 1) / 2, n1 = (m.nel[1] - c1 + 1) / 2;
  const int n2 = D == 3 ? (m.nel[2] - c2 + 1) / 2 : 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_el_c = n0 * n1 * n2;
  if (t >= n_el_c * NEN * NEN) return;
  const int ke = t / (NEN * NEN), I = (t / NEN) % NEN, J = t % NEN;
  const int kx = ke % n0, ky = (ke / n0) % n1, kz = ke / (n0 * n1);
  const int ex = 2 * kx + c0, ey = 2 * ky + c1, ez = D == 3 ? 2 * kz + c2 : 0;
  const int e = ex + m.nel[0] * (ey + m.nel[1] * ez);
  double omega = 1.0;
#pragma unroll
  for (int k = 0; k < D; ++k) omega *= 0.5 * m.h[k];
  double Kb[D][D];
  double fb[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    fb[i] = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) Kb[i][k] = 0.0;
  }
  for (int g = 0; g < NQ; ++g) {
    const int q = e * NQ + g;
    double gI[3], gJ[3];
    grad_N<D>(I, g, m, gI);
    grad_N<D>(J, g, m, gJ);
    if (m.A) {
      const double* A = m.A + (size_t)q * D * D * D * D;
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          double s = 0.0;
#pragma unroll
          for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b) s += gI[a] * A[((i * D + a) * D + k) * D + b] * gJ[b];
          Kb[i][k] += omega * s;
        }
    }
    if (J == 0) {
      const double* P = m.P + (size_t)q * D * D;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) s += P[i * D + a] * gI[a];
        fb[i] += omega * s;
      }
    }
  }
  const int nodeI = corner_node<D>(e, I, m);
  if (J == 0) {
#pragma unroll
    for (int i = 0; i < D; ++i) m.f[(size_t)nodeI * D + i] += fb[i];
  }
  if (m.A) {
    const int base = m.blk_base[((size_t)e * NEN + I) * NEN + J];
    const int stride = m.blk_stride[(size_t)e * NEN + I];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int k = 0; k < D; ++k) m.K[base + i * stride + k] += Kb[i][k];
  }
}

// u[dof_k] = scale * value_k on the Dirichlet dofs; du <- 0 everywhere (start of a load step)
__global__ void macro_dirichlet_kernel(double* u, double* du, int n, const int32_t* dofs, const double* vals,
                                       int n_fixed, double scale) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_fixed) u[dofs[t]] = scale * vals[t];
  if (du)
    for (int i = t; i < n; i += gridDim.x * blockDim.x) du[i] = 0.0;
}

// u += du (du is zero on the Dirichlet dofs)
__global__ void macro_update_kernel(double* u, const double* du, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) u[t] += du[t];
}

// y = scale K x over all rows (CSR; 8 lanes per row, 4 rows per warp, shuffle sum).  The loop
// bound is uniform over each warp (its 4 rows share `base`), so the shuffles see all lanes.
__global__ void macro_spmv_kernel(const int32_t* rowptr, const int32_t* col, const double* K, const double* x,
                                  double scale, double* y, int n) {
  const int lane8 = threadIdx.x & 7, sub = (threadIdx.x & 31) >> 3;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, warps = (gridDim.x * blockDim.x) >> 5;
  for (int base = 4 * warp; base < n; base += 4 * warps) {
    const int i = base + sub;
    double s = 0.0;
    if (i < n)
      for (int k = rowptr[i] + lane8; k < rowptr[i + 1]; k += 8) s = fma(K[k], x[col[k]], s);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (lane8 == 0 && i < n) y[i] = scale * s;
  }
}

}  // namespace

cudaError_t macro_spmv_launch(const int32_t* rowptr, const int32_t* col, const double* K, const double* x,
                              double scale, double* y, int n, cudaStream_t stream) {
  const int threads = 256, rows_per_block = threads / 8;
  int blocks = (n + rows_per_block - 1) / rows_per_block;
  blocks = blocks < 1 ? 1 : (blocks > 1024 ? 1024 : blocks);
  macro_spmv_kernel<<<blocks, threads, 0, stream>>>(rowptr, col, K, x, scale, y, n);
  return cudaGetLastError();
}

cudaError_t macro_dirichlet_launch(double* u, double* du, int n, const int32_t* dofs, const double* vals, int n_fixed,
                                   double scale, cudaStream_t stream) {
  const int work = n_fixed > 0 ? n_fixed : 1;
  const int blocks = (work + 255) / 256 > 0 ? (work + 255) / 256 : 1;
  macro_dirichlet_kernel<<<blocks < 64 ? 64 : blocks, 256, 0, stream>>>(u, du, n, dofs, vals, n_fixed, scale);
  return cudaGetLastError();
}

cudaError_t macro_update_launch(double* u, const double* du, int n, cudaStream_t stream) {
  macro_update_kernel<<<(n + 255) / 256, 256, 0, stream>>>(u, du, n);
  return cudaGetLastError();
}

cudaError_t macro_qp_F_launch(const MacroArgs& m, cudaStream_t stream) {
  const int threads = 128, blocks = (m.n_qp + threads - 1) / threads;
  if (m.dim == 2)
    macro_qp_F_kernel<2><<<blocks, threads, 0, stream>>>(m);
  else
    macro_qp_F_kernel<3><<<blocks, threads, 0, stream>>>(m);
  return cudaGetLastError();
}

cudaError_t macro_assemble_launch(const MacroArgs& m, cudaStream_t stream, int* launches) {
  const int ncol = 1 << m.dim, nen = 1 << m.dim;
  for (int c = 0; c < ncol; ++c) {
    const int c0 = c & 1, c1 = (c >> 1) & 1, c2 = (c >> 2) & 1;
    const int n0 = (m.nel[0] - c0 + 1) / 2, n1 = (m.nel[1] - c1 + 1) / 2;
    const int n2 = m.dim == 3 ? (m.nel[2] - c2 + 1) / 2 : 1;
    const int total = n0 * n1 * n2 * nen * nen;
    if (total <= 0) continue;
    const int threads = 128, blocks = (total + threads - 1) / threads;
    if (m.dim == 2)
      macro_assemble_kernel<2><<<blocks, threads, 0, stream>>>(m, c);
    else
      macro_assemble_kernel<3><<<blocks, threads, 0, stream>>>(m, c);
    ++*launches;
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

}  // namespace fehmm
