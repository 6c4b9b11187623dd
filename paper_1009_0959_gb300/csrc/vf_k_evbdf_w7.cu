// Generalised entropy vector filter with the angular distance (Sec. 3.3 with
// the angle of Sec. 3.1): 7 x 7 window kernels.
#include "vf_launch.cuh"

namespace vf {
cudaError_t launch_evbdf_w7(const Launch& L, int approx, int degree, int ty, int grid,
                            cudaStream_t s) {
  return launch_apx<7, kEVBDF>(L, approx, degree, ty, grid, s);
}
}  // namespace vf
