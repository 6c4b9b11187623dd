// AMNF with the Gaussian kernel (Sec. 3.2, Eq. equ_amnf): 5 x 5 window kernels.
#include "vf_launch.cuh"

namespace vf {
cudaError_t launch_amnfg_w5(const Launch& L, int approx, int degree, int ty, int grid,
                          cudaStream_t s) {
  return launch_apx<5, kAMNFG>(L, approx, degree, ty, grid, s);
}
}  // namespace vf
