// Gated window filters, 7 x 7 window.
#include "vf_gated.cuh"

namespace vf {
cudaError_t launch_gated_w7(const Launch& L, const uint8_t* flags, long long flag_pitch,
                             int crit, int apx, int degree, int ty, int grid, cudaStream_t s) {
  return launch_gated_w<7>(L, GateFlags{flags, flag_pitch}, crit, apx, degree, ty, grid, s);
}
cudaError_t launch_sparse_w7(const Launch& L, const int* list, const unsigned* count,
                              unsigned limit, int sms, int crit, int apx, int degree,
                              cudaStream_t s) {
  return launch_sparse_w<7>(L, list, count, limit, sms, crit, apx, degree, s);
}
}  // namespace vf
