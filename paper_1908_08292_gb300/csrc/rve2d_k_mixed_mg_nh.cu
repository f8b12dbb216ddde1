// 2D RVE kernel instantiation: mixed precision, multigrid, neo-Hookean.
#include "rve2d.cuh"

namespace fehmm {
cudaError_t rve2d_launch_mixed_mg_nh(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream) {
  return rve2d_launch_instance<float, false, true, 0>(a, n_blocks, smem, stream);
}
}  // namespace fehmm
