// Entropy vector median filter (Sec. 3.3, Eq. equ_evf): 3 x 3 window kernels.
#include "vf_launch.cuh"

namespace vf {
cudaError_t launch_evmf_w3(const Launch& L, int approx, int degree, int ty, int grid,
                          cudaStream_t s) {
  return launch_apx<3, kEVMF>(L, approx, degree, ty, grid, s);
}
}  // namespace vf
