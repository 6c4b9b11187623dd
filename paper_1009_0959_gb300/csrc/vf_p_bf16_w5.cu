// Packed bf16 x 2 window kernels, 5 x 5 window.
#include "vf_packed_launch.cuh"

namespace vf {
cudaError_t launch_packed_bf16_w5(const Launch& L, int crit, int apx, int degree, int ty,
                                  int grid, cudaStream_t s) {
  return launch_packed_w<5, __nv_bfloat162>(L, crit, apx, degree, ty, grid, s);
}
}  // namespace vf
