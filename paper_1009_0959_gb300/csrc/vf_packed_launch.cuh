// vf_packed_launch.cuh -- launch helper of the packed-precision kernels.
#pragma once

#include "vf_packed.cuh"

namespace vf {

template <int W, int CRIT, int APX, int DEG, class T>
cudaError_t launch_packed_one(const Launch& L, int ty, int grid, cudaStream_t s) {
  const size_t smem = packed_smem_bytes(W, ty);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(packed_kernel<W, CRIT, APX, DEG, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return launch_maybe_pdl(L.pdl != 0, packed_kernel<W, CRIT, APX, DEG, T>, dim3(grid),
                          dim3(kTX * ty), smem, s, L);
}

// One window size and format.  The per-sample approximants of AMNF and EVMF run
// as degree 6 with zero-padded coefficients (bit-identical to the exact
// degree); the BVDF pair-term polynomial keeps its degree as a template.
template <int W, class T>
cudaError_t launch_packed_w(const Launch& L, int crit, int apx, int degree, int ty, int grid,
                            cudaStream_t s) {
  switch (crit) {
    case kVMF: return launch_packed_one<W, kVMF, kExact, 0, T>(L, ty, grid, s);
    case kBVDF:
      if (apx != kPoly) return cudaErrorInvalidValue;
      switch (degree) {
        case 2: return launch_packed_one<W, kBVDF, kPoly, 2, T>(L, ty, grid, s);
        case 3: return launch_packed_one<W, kBVDF, kPoly, 3, T>(L, ty, grid, s);
        case 4: return launch_packed_one<W, kBVDF, kPoly, 4, T>(L, ty, grid, s);
        case 5: return launch_packed_one<W, kBVDF, kPoly, 5, T>(L, ty, grid, s);
        case 6: return launch_packed_one<W, kBVDF, kPoly, 6, T>(L, ty, grid, s);
        default: return cudaErrorInvalidValue;
      }
    case kAMNFE:
      if (apx == kExact) return launch_packed_one<W, kAMNFE, kExact, 0, T>(L, ty, grid, s);
      if (apx == kPoly) return launch_packed_one<W, kAMNFE, kPoly, 6, T>(L, ty, grid, s);
      return launch_packed_one<W, kAMNFE, kRational, 4, T>(L, ty, grid, s);
    case kAMNFG:
      if (apx == kExact) return launch_packed_one<W, kAMNFG, kExact, 0, T>(L, ty, grid, s);
      if (apx == kPoly) return launch_packed_one<W, kAMNFG, kPoly, 6, T>(L, ty, grid, s);
      return launch_packed_one<W, kAMNFG, kRational, 4, T>(L, ty, grid, s);
    case kEVMF:
      if (apx == kExact) return launch_packed_one<W, kEVMF, kExact, 0, T>(L, ty, grid, s);
      if (apx == kPoly) return launch_packed_one<W, kEVMF, kPoly, 6, T>(L, ty, grid, s);
      return launch_packed_one<W, kEVMF, kRational, 4, T>(L, ty, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace vf
