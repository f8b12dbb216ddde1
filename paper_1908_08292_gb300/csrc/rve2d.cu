// Host side of the 2D batched periodic-RVE solver: shared-memory and scratch sizes and the
// dispatch to the kernel instantiations.  Each instantiation is compiled in a translation unit
// of its own (rve2d_k_*.cu) so that the builds run in parallel; the device code is rve2d.cuh.
#include "rve2d.cuh"

namespace fehmm {

cudaError_t rve2d_launch_mixed_mg_nh(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream);
cudaError_t rve2d_launch_mixed_mg_svk(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream);
cudaError_t rve2d_launch_mixed_bj_nh(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream);
cudaError_t rve2d_launch_mixed_bj_svk(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream);
cudaError_t rve2d_launch_fp64_mg_nh(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream);
cudaError_t rve2d_launch_fp64_mg_svk(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream);
cudaError_t rve2d_launch_fp64_bj_nh(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream);
cudaError_t rve2d_launch_fp64_bj_svk(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream);
cudaError_t rve2d_launch_fp64_fixed_nh(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream);

size_t rve2d_smem_bytes(int nn_max, bool mixed) {
  return mixed ? smem2d_layout<float>(nn_max, nullptr, nullptr) : smem2d_layout<double>(nn_max, nullptr, nullptr);
}

long long rve2d_scratch_stride(int nn_max, bool mixed) {
  // mixed: staged element tangents [36][nn_max] and the coarse element matrices of the multigrid;
  // FP64: stencil and staged tangents [72][nn_max], then the whole multigrid
  return mixed ? 36LL * nn_max + mg_slow_max(nn_max) : 72LL * nn_max + mg_fast_max(nn_max) + mg_slow_max(nn_max);
}

size_t rve2d_scratch_bytes(int nn_max, bool mixed, int n_blocks) {
  return (mixed ? sizeof(float) : sizeof(double)) * (size_t)rve2d_scratch_stride(nn_max, mixed) * n_blocks;
}

int rve2d_threads() { return kThreads2D; }

// The multigrid and block-Jacobi paths and the two laws are separate instantiations, so each is
// register-allocated on its own.
cudaError_t rve2d_launch(const Rve2dArgs& a, bool mixed, int n_blocks, cudaStream_t stream) {
  const size_t smem = rve2d_smem_bytes(a.nn_max, mixed);
  const bool svk = a.law == 1;
  if (mixed) {
    if (a.mg) return svk ? rve2d_launch_mixed_mg_svk(a, n_blocks, smem, stream) : rve2d_launch_mixed_mg_nh(a, n_blocks, smem, stream);
    return svk ? rve2d_launch_mixed_bj_svk(a, n_blocks, smem, stream) : rve2d_launch_mixed_bj_nh(a, n_blocks, smem, stream);
  }
  if (a.mg) return svk ? rve2d_launch_fp64_mg_svk(a, n_blocks, smem, stream) : rve2d_launch_fp64_mg_nh(a, n_blocks, smem, stream);
  return svk ? rve2d_launch_fp64_bj_svk(a, n_blocks, smem, stream) : rve2d_launch_fp64_bj_nh(a, n_blocks, smem, stream);
}

cudaError_t rve2d_launch_fixed_fp64(const Rve2dArgs& a, int n_blocks, cudaStream_t stream) {
  return rve2d_launch_fp64_fixed_nh(a, n_blocks, rve2d_smem_bytes(a.nn_max, false), stream);
}

}  // namespace fehmm
