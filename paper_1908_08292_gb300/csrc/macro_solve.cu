// Macro Newton correction: K_ff du_f = -f_f with du = 0 on the Dirichlet dofs (the linearised
// macro problem, Eq. L(GH) with the tangent of Eq. ModifiedBilinearForm-3 assembled as in
// Eq. Assem_k_T_IK_mac).  Jacobi-preconditioned CG in FP64 over the CSR tangent, run as one
// cooperative launch (1024-thread blocks, about 64k nonzeros each, at most one per SM, all
// co-resident; grid-wide barriers between the
// sparse product, the inner products and the vector updates).  The inner products are summed
// per block, then every block adds the block partials in the same order, so all blocks take
// the same decisions.  The first output is |f_free|_2, the macro convergence measure.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rve_args.h"

namespace cg = cooperative_groups;

namespace fehmm {
namespace {

constexpr int kSolveThreads = 1024;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid-wide sum of one value per thread (every block returns the same total).
__device__ double grid_sum(double v, double* partial, double* sbuf, cg::grid_group& grid) {
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sbuf[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kSolveThreads / 32; ++w) s += sbuf[w];
    partial[blockIdx.x] = s;
  }
  grid.sync();
  double t = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b) t += partial[b];  // same order in every block
  __syncthreads();  // sbuf reused by the next call
  return t;
}

__global__ void __launch_bounds__(kSolveThreads) macro_pcg_kernel(const MacroSolveArgs a) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double sbuf[kSolveThreads / 32];
  const int n = a.n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  double* x = a.du;
  double* r = a.work;
  double* z = a.work + n;
  double* p = a.work + 2 * (size_t)n;
  double* q = a.work + 3 * (size_t)n;
  double* dg = a.work + 4 * (size_t)n;        // Jacobi diagonal
  double* partial = a.work + 5 * (size_t)n;  // [gridDim.x]
  double* partial2 = partial + gridDim.x;     // second buffer: alternate between reductions
  // diagonal for the Jacobi preconditioner
  double ff = 0.0, rz = 0.0;
  for (int i = tid; i < n; i += stride) {
    const bool fixed = a.fixed[i] != 0;
    double d = 1.0;
    for (int k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k)
      if (a.col[k] == i) d = a.K[k];
    dg[i] = d;
    const double ri = fixed ? 0.0 : -a.f[i];
    x[i] = 0.0;
    r[i] = ri;
    z[i] = fixed ? 0.0 : ri / d;
    p[i] = z[i];
    ff += ri * ri;
    rz += ri * z[i];
  }
  const double fnorm2 = grid_sum(ff, partial, sbuf, grid);
  rz = grid_sum(rz, partial2, sbuf, grid);
  if (tid == 0) a.out[0] = sqrt(fnorm2);
  const double rz0 = rz;
  int it = 0;
  int status = 0;
  if (rz0 > 0.0) {
    const double stop = a.rtol * a.rtol * rz0;
    for (;;) {
      if (it >= a.max_it) {
        status = 1;
        break;
      }
      double pq = 0.0;
      for (int i = tid; i < n; i += stride) {
        double s = 0.0;
        if (!a.fixed[i])
          for (int k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k) s += a.K[k] * p[a.col[k]];
        q[i] = s;
        pq += p[i] * s;
      }
      pq = grid_sum(pq, partial, sbuf, grid);
      if (!(pq > 0.0)) {
        status = 2;
        break;
      }
      const double alpha = rz / pq;
      double rzn = 0.0;
      for (int i = tid; i < n; i += stride) {
        if (a.fixed[i]) continue;
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
        z[i] = r[i] / dg[i];
        rzn += r[i] * z[i];
      }
      rzn = grid_sum(rzn, partial2, sbuf, grid);
      ++it;
      if (rzn <= stop) break;
      const double beta = rzn / rz;
      rz = rzn;
      for (int i = tid; i < n; i += stride) p[i] = z[i] + beta * p[i];
      grid.sync();
    }
  }
  if (tid == 0) {
    a.out[1] = (double)it;
    a.out[2] = (double)status;
  }
}

}  // namespace

size_t macro_solve_work_doubles(int n, int blocks) { return 5 * (size_t)n + 2 * (size_t)blocks; }

// Blocks for the cooperative solve: about 64k nonzeros per block (grid-wide barriers get more
// expensive with every block, the sparse product needs enough of them), at most one per SM.
int macro_solve_blocks(int num_sms, long long nnz) {
  long long b = (nnz + 65535) / 65536;
  if (b < 1) b = 1;
  return (int)(b < num_sms ? b : num_sms);
}

cudaError_t macro_solve_launch(const MacroSolveArgs& a, int blocks, cudaStream_t stream) {
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((void*)macro_pcg_kernel, dim3(blocks), dim3(kSolveThreads), args, 0, stream);
}

}  // namespace fehmm
