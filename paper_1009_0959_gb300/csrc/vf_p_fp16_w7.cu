// Packed fp16 x 2 window kernels, 7 x 7 window.
#include "vf_packed_launch.cuh"

namespace vf {
cudaError_t launch_packed_fp16_w7(const Launch& L, int crit, int apx, int degree, int ty,
                                  int grid, cudaStream_t s) {
  return launch_packed_w<7, __half2>(L, crit, apx, degree, ty, grid, s);
}
}  // namespace vf
