// 2D RVE kernel instantiation: FP64, block-Jacobi, fixed single-grid layout (no-allocation entry).
#include "rve2d.cuh"

namespace fehmm {
cudaError_t rve2d_launch_fp64_fixed(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream) {
  return rve2d_launch_instance<double, true, false>(a, n_blocks, smem, stream);
}
}  // namespace fehmm
