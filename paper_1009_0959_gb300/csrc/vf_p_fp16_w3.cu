// Packed fp16 x 2 window kernels, 3 x 3 window.
#include "vf_packed_launch.cuh"

namespace vf {
cudaError_t launch_packed_fp16_w3(const Launch& L, int crit, int apx, int degree, int ty,
                                  int grid, cudaStream_t s) {
  return launch_packed_w<3, __half2>(L, crit, apx, degree, ty, grid, s);
}
}  // namespace vf
