// AMNF with the Gaussian kernel (Sec. 3.2, Eq. equ_amnf): 3 x 3 window kernels.
#include "vf_launch.cuh"

namespace vf {
cudaError_t launch_amnfg_w3(const Launch& L, int approx, int degree, int ty, int grid,
                          cudaStream_t s) {
  return launch_apx<3, kAMNFG>(L, approx, degree, ty, grid, s);
}
}  // namespace vf
