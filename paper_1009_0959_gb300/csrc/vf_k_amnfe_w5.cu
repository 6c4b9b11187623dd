// AMNF with the exponential kernel (Sec. 3.2, Eq. equ_amnf): 5 x 5 window kernels.
#include "vf_launch.cuh"

namespace vf {
cudaError_t launch_amnfe_w5(const Launch& L, int approx, int degree, int ty, int grid,
                          cudaStream_t s) {
  return launch_apx<5, kAMNFE>(L, approx, degree, ty, grid, s);
}
}  // namespace vf
