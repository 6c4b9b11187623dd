// Pair-reuse window kernels, 5 x 5: EVMF (the entropy switch per output
// in the finish phase, the vector median from the Euclidean aggregates).
#include "vf_reuse.cuh"

namespace vf {
cudaError_t launch_reuse_evmf_w5(const Launch& L, int apx, int degree, int grid, cudaStream_t s) {
  return launch_reuse_evmf<5>(L, apx, degree, grid, s);
}
}  // namespace vf
