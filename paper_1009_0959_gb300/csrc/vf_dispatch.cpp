// vf_dispatch.cpp -- criterion x window dispatch to the kernel translation units.
#include "vf_internal.h"

namespace vf {

#define VF_CASE(name)                                                     \
  switch (w) {                                                            \
    case 3: return launch_##name##_w3(L, approx, degree, ty, grid, s);    \
    case 5: return launch_##name##_w5(L, approx, degree, ty, grid, s);    \
    case 7: return launch_##name##_w7(L, approx, degree, ty, grid, s);    \
    default: return cudaErrorInvalidValue;                                \
  }

cudaError_t launch_filter(const Launch& L, int criterion, int w, int approx, int degree, int ty,
                          int grid, cudaStream_t s) {
  switch (criterion) {
    case kVMF: VF_CASE(vmf)
    case kBVDF: VF_CASE(bvdf)
    case kAMNFE: VF_CASE(amnfe)
    case kAMNFG: VF_CASE(amnfg)
    case kEVMF: VF_CASE(evmf)
    case kEVBDF: VF_CASE(evbdf)
    default: return cudaErrorInvalidValue;
  }
}

#undef VF_CASE

cudaError_t launch_reuse(const Launch& L, int crit, int w, int apx, int degree, int grid,
                         cudaStream_t s) {
  const bool amnf = crit == kAMNFE || crit == kAMNFG;
  if (crit == kEVMF) {
    if (w == 3) return launch_reuse_evmf_w3(L, apx, degree, grid, s);
    if (w == 5) return launch_reuse_evmf_w5(L, apx, degree, grid, s);
    if (w == 7) return launch_reuse_evmf_w7(L, apx, degree, grid, s);
    return cudaErrorInvalidValue;
  }
  if (w == 3) return amnf ? launch_reuse_amnf_w3(L, crit, apx, degree, grid, s)
                          : launch_reuse_sel_w3(L, crit, apx, degree, grid, s);
  if (w == 5) return amnf ? launch_reuse_amnf_w5(L, crit, apx, degree, grid, s)
                          : launch_reuse_sel_w5(L, crit, apx, degree, grid, s);
  if (w == 7) return amnf ? launch_reuse_amnf_w7(L, crit, apx, degree, grid, s)
                          : launch_reuse_sel_w7(L, crit, apx, degree, grid, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_packed(const Launch& L, int precision, int criterion, int w, int approx,
                          int degree, int ty, int grid, cudaStream_t s) {
  if (precision == 1) {
    if (w == 3) return launch_packed_fp16_w3(L, criterion, approx, degree, ty, grid, s);
    if (w == 5) return launch_packed_fp16_w5(L, criterion, approx, degree, ty, grid, s);
    if (w == 7) return launch_packed_fp16_w7(L, criterion, approx, degree, ty, grid, s);
  } else if (precision == 2) {
    if (w == 3) return launch_packed_bf16_w3(L, criterion, approx, degree, ty, grid, s);
    if (w == 5) return launch_packed_bf16_w5(L, criterion, approx, degree, ty, grid, s);
    if (w == 7) return launch_packed_bf16_w7(L, criterion, approx, degree, ty, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace vf
