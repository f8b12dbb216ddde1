// 2D RVE kernel instantiation: FP64, block-Jacobi, St. Venant-Kirchhoff.
#include "rve2d.cuh"

namespace fehmm {
cudaError_t rve2d_launch_fp64_bj_svk(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream) {
  return rve2d_launch_instance<double, false, false, 1>(a, n_blocks, smem, stream);
}
}  // namespace fehmm
