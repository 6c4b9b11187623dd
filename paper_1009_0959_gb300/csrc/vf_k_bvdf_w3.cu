// Basic vector directional filter (Sec. 3.1), exact and piecewise minimax arccos: 3 x 3 window kernels.
#include "vf_launch.cuh"

namespace vf {
cudaError_t launch_bvdf_w3(const Launch& L, int approx, int degree, int ty, int grid,
                          cudaStream_t s) {
  return launch_apx<3, kBVDF>(L, approx, degree, ty, grid, s);
}
}  // namespace vf
