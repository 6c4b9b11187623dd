// Pair-reuse window kernels, 5 x 5: AMNFE and AMNFG.
#include "vf_reuse.cuh"

namespace vf {
cudaError_t launch_reuse_amnf_w5(const Launch& L, int crit, int apx, int degree, int grid,
                                  cudaStream_t s) {
  return launch_reuse_amnf<5>(L, crit, apx, degree, grid, s);
}
}  // namespace vf
