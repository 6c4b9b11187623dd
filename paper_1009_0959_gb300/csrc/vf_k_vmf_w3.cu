// Vector median filter (Sec. 3.3, first branch of Eq. equ_evf): 3 x 3 window kernels.
#include "vf_launch.cuh"

namespace vf {
cudaError_t launch_vmf_w3(const Launch& L, int approx, int degree, int ty, int grid,
                          cudaStream_t s) {
  return launch_apx<3, kVMF>(L, approx, degree, ty, grid, s);
}
}  // namespace vf
