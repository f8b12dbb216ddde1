// Macro Newton correction: K_ff du_f = -f_f with du = 0 on the Dirichlet dofs (the linearised
// macro problem, Eq. L(GH) with the tangent of Eq. ModifiedBilinearForm-3 assembled as in
// Eq. Assem_k_T_IK_mac).  Jacobi-preconditioned CG in FP64 over the CSR tangent.
//
// One cooperative launch, one block per SM at most, all co-resident.  The CG is the single-
// reduction form of Chronopoulos and Gear: per iteration the vector updates and u = M^-1 r (one
// thread per row), a grid barrier (u visible), the sparse product w = K u (8 lanes per row,
// strided nonzeros per lane, shuffle sum) together with the partial inner products
// gamma = r.u and delta = w.u, and a second grid barrier after which every block adds the block
// partials in the same order — two grid barriers per iteration and identical decisions in
// every block.  Fixed rows carry M^-1 = 0 and no product, which keeps their r, u, p, x at zero.
// The first output is |f_free|_2, the macro convergence measure.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rve_args.h"

namespace cg = cooperative_groups;

namespace fehmm {
namespace {

constexpr int kSolveThreads = 256;
constexpr int kRowLanes = 8;                              // lanes per matrix row in the product
constexpr int kRowsPerWarp = 32 / kRowLanes;              // 4
constexpr int kRowsPerBlock = kSolveThreads / kRowLanes;  // 32

// Sum (a, b) over the grid: block sums -> partial[2*block], grid barrier, every block adds the
// partials in index order (warp 0, fixed shuffle tree), so all blocks get identical totals.
// Consecutive calls must use alternate partial buffers: a block may write the next call's
// partials while a slower block still reads this call's, and only a grid barrier of the call
// in between (every call has one) orders the reads of call k before the writes of call k + 2.
__device__ void grid_sum2(double& a, double& b, double* partial, double (*sbuf)[2], cg::grid_group& grid) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sbuf[warp][0] = a;
    sbuf[warp][1] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int k = 0; k < kSolveThreads / 32; ++k) {
      s0 += sbuf[k][0];
      s1 += sbuf[k][1];
    }
    partial[2 * blockIdx.x] = s0;
    partial[2 * blockIdx.x + 1] = s1;
  }
  grid.sync();
  if (warp == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int j = lane; j < (int)gridDim.x; j += 32) {
      t0 += partial[2 * j];
      t1 += partial[2 * j + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      t0 += __shfl_xor_sync(0xffffffffu, t0, o);
      t1 += __shfl_xor_sync(0xffffffffu, t1, o);
    }
    if (lane == 0) {
      sbuf[0][0] = t0;
      sbuf[0][1] = t1;
    }
  }
  __syncthreads();
  a = sbuf[0][0];
  b = sbuf[0][1];
  __syncthreads();  // sbuf is reused by the next call
}

// w = K u over this block's rows (8 lanes per row); returns this thread's share of w.u.  The
// loop bound is uniform over each warp (its 4 rows share `base`), so the shuffles see all lanes.
__device__ __forceinline__ double spmv_rows(const MacroSolveArgs& a, const double* dinv, const double* u, double* w,
                                            int n) {
  const int lane8 = threadIdx.x % kRowLanes;
  const int warp_rows = (blockIdx.x * kSolveThreads + (threadIdx.x & ~31)) / kRowLanes;  // first row of the warp
  const int sub = (threadIdx.x & 31) / kRowLanes;
  const int n_rows_grid = gridDim.x * kRowsPerBlock;
  double wu = 0.0;
  for (int base = warp_rows; base < n; base += n_rows_grid) {
    const int i = base + sub;
    double s = 0.0;
    if (i < n && dinv[i] != 0.0) {
      const int k1 = a.rowptr[i + 1];
      for (int k = a.rowptr[i] + lane8; k < k1; k += kRowLanes) s = fma(a.K[k], u[a.col[k]], s);
    }
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (lane8 == 0 && i < n) {
      w[i] = s;
      wu = fma(s, u[i], wu);
    }
  }
  return wu;
}

__global__ void __launch_bounds__(kSolveThreads) macro_pcg_kernel(const MacroSolveArgs a) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double sbuf[kSolveThreads / 32][2];
  const int n = a.n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  double* x = a.du;
  double* r = a.work;
  double* u = r + n;
  double* w = u + n;
  double* p = w + n;
  double* s = p + n;
  double* dinv = s + n;
  double* partials = dinv + n;  // two buffers of [2 * gridDim.x], alternated between grid sums
  int parity = 0;
  auto next_partial = [&]() {
    double* buf = partials + (size_t)parity * 2 * gridDim.x;
    parity ^= 1;
    return buf;
  };
  // Jacobi diagonal, r = -f on free rows, u = M^-1 r
  double ff = 0.0, ru = 0.0;
  for (int i = tid; i < n; i += stride) {
    const bool fixed = a.fixed[i] != 0;
    double d = 1.0;
    for (int k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k)
      if (a.col[k] == i) d = a.K[k];
    const double di = fixed ? 0.0 : 1.0 / d;
    const double ri = fixed ? 0.0 : -a.f[i];
    dinv[i] = di;
    x[i] = 0.0;
    r[i] = ri;
    u[i] = ri * di;
    p[i] = 0.0;
    s[i] = 0.0;
    ff = fma(ri, ri, ff);
    ru = fma(ri, ri * di, ru);
  }
  grid_sum2(ff, ru, next_partial(), sbuf, grid);  // its grid barrier also publishes u and dinv
  if (tid == 0) a.out[0] = sqrt(ff);
  double gamma = ru;
  const double stop = a.rtol * a.rtol * gamma;
  int it = 0, status = 0;
  if (gamma > 0.0) {
    double delta = spmv_rows(a, dinv, u, w, n), unused = 0.0;
    grid_sum2(delta, unused, next_partial(), sbuf, grid);
    double alpha = gamma / delta, beta = 0.0;
    if (!(delta > 0.0)) status = 2;
    while (status == 0) {
      // p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = M^-1 r, gamma' = r.u
      double g = 0.0;
      for (int i = tid; i < n; i += stride) {
        const double pi = fma(beta, p[i], u[i]);
        const double si = fma(beta, s[i], w[i]);
        p[i] = pi;
        s[i] = si;
        x[i] = fma(alpha, pi, x[i]);
        const double ri = fma(-alpha, si, r[i]);
        r[i] = ri;
        const double ui = ri * dinv[i];
        u[i] = ui;
        g = fma(ri, ui, g);
      }
      ++it;
      grid.sync();  // u complete before the product
      double d = spmv_rows(a, dinv, u, w, n);
      grid_sum2(g, d, next_partial(), sbuf, grid);
      if (g <= stop) break;
      if (it >= a.max_it) {
        status = 1;
        break;
      }
      beta = g / gamma;
      const double den = d - beta * g / alpha;
      if (!(den > 0.0)) {
        status = 2;
        break;
      }
      alpha = g / den;
      gamma = g;
    }
  }
  if (tid == 0) {
    a.out[1] = (double)it;
    a.out[2] = (double)status;
  }
}

}  // namespace

size_t macro_solve_work_doubles(int n, int blocks) { return 6 * (size_t)n + 4 * (size_t)blocks; }

// One block per 32 rows (one pass of the product), at most one per SM.
int macro_solve_blocks(int num_sms, long long n_rows) {
  long long b = (n_rows + kRowsPerBlock - 1) / kRowsPerBlock;
  if (b < 1) b = 1;
  return (int)(b < num_sms ? b : num_sms);
}

cudaError_t macro_solve_launch(const MacroSolveArgs& a, int blocks, cudaStream_t stream) {
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((void*)macro_pcg_kernel, dim3(blocks), dim3(kSolveThreads), args, 0, stream);
}

}  // namespace fehmm
