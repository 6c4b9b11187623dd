// Pair-reuse window kernels, 3 x 3: VMF and BVDF.
#include "vf_reuse.cuh"

namespace vf {
cudaError_t launch_reuse_sel_w3(const Launch& L, int crit, int apx, int degree, int grid,
                                 cudaStream_t s) {
  return launch_reuse_sel<3>(L, crit, apx, degree, grid, s);
}
}  // namespace vf
