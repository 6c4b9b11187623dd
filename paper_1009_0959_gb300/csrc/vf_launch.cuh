// vf_launch.cuh -- launch helper shared by the per-criterion translation units.
#pragma once

#include "vf_evmf.cuh"
#include "vf_kernels.cuh"

namespace vf {

template <int W, int CRIT, int APX, int DEG>
cudaError_t launch_one(const Launch& L, int ty, int grid, cudaStream_t s) {
  // EVMF 5 x 5: persistent kernel with a work queue (measured: for w = 3 the
  // 36-pair median is too cheap for the queue copies to pay; for w = 7 the
  // 196-byte entries and the shared-memory aggregate slots leave two CTAs per
  // SM, and the one-tile kernel is 20 % faster)
  if constexpr (CRIT == kEVMF && W == 5) {
    return launch_evmf_queue<W, APX, DEG>(L, ty, grid, s);
  } else if constexpr (outputs_per_thread(W, CRIT) == 2) {
    // 32 x ty threads, 32 x 2ty outputs
    const size_t smem = smem_bytes(W, CRIT, 2 * ty);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(filter2_kernel<W, CRIT, APX, DEG>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    return launch_maybe_pdl(L.pdl != 0, filter2_kernel<W, CRIT, APX, DEG>, dim3(grid),
                            dim3(kTX * ty), smem, s, L);
  } else {
    const size_t smem = smem_bytes(W, CRIT, ty);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(filter_kernel<W, CRIT, APX, DEG>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    return launch_maybe_pdl(L.pdl != 0, filter_kernel<W, CRIT, APX, DEG>, dim3(grid),
                            dim3(kTX * ty), smem, s, L);
  }
}

// Polynomial degree 2..6 as a template argument.
template <int W, int CRIT, int APX>
cudaError_t launch_deg(const Launch& L, int degree, int ty, int grid, cudaStream_t s) {
  switch (degree) {
    case 2: return launch_one<W, CRIT, APX, 2>(L, ty, grid, s);
    case 3: return launch_one<W, CRIT, APX, 3>(L, ty, grid, s);
    case 4: return launch_one<W, CRIT, APX, 4>(L, ty, grid, s);
    case 5: return launch_one<W, CRIT, APX, 5>(L, ty, grid, s);
    case 6: return launch_one<W, CRIT, APX, 6>(L, ty, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

// exact / polynomial (any degree) / rational for one window size.
template <int W, int CRIT>
cudaError_t launch_apx(const Launch& L, int approx, int degree, int ty, int grid, cudaStream_t s) {
  switch (approx) {
    case kExact: return launch_one<W, CRIT, kExact, 0>(L, ty, grid, s);
    case kPoly: return launch_deg<W, CRIT, kPoly>(L, degree, ty, grid, s);
    case kRational:
      if constexpr (CRIT == kBVDF || CRIT == kEVBDF) return cudaErrorInvalidValue;
      else return launch_one<W, CRIT, kRational, 4>(L, ty, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace vf
