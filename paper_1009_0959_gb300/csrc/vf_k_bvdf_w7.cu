// Basic vector directional filter (Sec. 3.1), exact and piecewise minimax arccos: 7 x 7 window kernels.
#include "vf_launch.cuh"

namespace vf {
cudaError_t launch_bvdf_w7(const Launch& L, int approx, int degree, int ty, int grid,
                          cudaStream_t s) {
  return launch_apx<7, kBVDF>(L, approx, degree, ty, grid, s);
}
}  // namespace vf
