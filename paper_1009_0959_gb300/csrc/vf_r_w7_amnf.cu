// Pair-reuse window kernels, 7 x 7: AMNFE and AMNFG.
#include "vf_reuse.cuh"

namespace vf {
cudaError_t launch_reuse_amnf_w7(const Launch& L, int crit, int apx, int degree, int grid,
                                  cudaStream_t s) {
  return launch_reuse_amnf<7>(L, crit, apx, degree, grid, s);
}
}  // namespace vf
