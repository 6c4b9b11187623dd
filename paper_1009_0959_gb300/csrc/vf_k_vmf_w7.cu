// Vector median filter (Sec. 3.3, first branch of Eq. equ_evf): 7 x 7 window kernels.
#include "vf_launch.cuh"

namespace vf {
cudaError_t launch_vmf_w7(const Launch& L, int approx, int degree, int ty, int grid,
                          cudaStream_t s) {
  return launch_apx<7, kVMF>(L, approx, degree, ty, grid, s);
}
}  // namespace vf
