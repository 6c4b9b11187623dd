// AMNF with the exponential kernel (Sec. 3.2, Eq. equ_amnf): 7 x 7 window kernels.
#include "vf_launch.cuh"

namespace vf {
cudaError_t launch_amnfe_w7(const Launch& L, int approx, int degree, int ty, int grid,
                          cudaStream_t s) {
  return launch_apx<7, kAMNFE>(L, approx, degree, ty, grid, s);
}
}  // namespace vf
