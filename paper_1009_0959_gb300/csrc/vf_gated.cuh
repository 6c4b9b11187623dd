// vf_gated.cuh -- the window filters restricted to the pixels a flag map
// marks (the learned gate's output); every other pixel is copied.  The flagged
// pixels of a tile are compacted in shared memory first, so the threads of a
// CTA work only on them (no divergence over copied pixels).
#pragma once

#include "vf_kernels.cuh"

namespace vf {

struct GateFlags {
  const uint8_t* flags;  // one byte per pixel, non-zero = filter
  long long pitch;
};

template <int W, int CRIT, int APX, int DEG>
__global__ void __launch_bounds__(256) gated_kernel(const __grid_constant__ Launch L,
                                                    const GateFlags G) {
  constexpr int R = W / 2;
  constexpr bool REG = uses_reg_path(W, CRIT);
  const int TY = blockDim.x / kTX;
  const TileSmem t = carve(W, REG, TY, blockDim.x);
  const int tile = blockIdx.x;
  const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
  const int x0 = txi * kTX, y0 = tyi * TY;
  __shared__ int s_count;
  if (threadIdx.x == 0) s_count = 0;
  stage_tile<CRIT, CRIT != kVMF>(L, t, x0, y0, R);
  __syncthreads();
  const int px = threadIdx.x % kTX, py = threadIdx.x / kTX;
  const int gx = x0 + px, gy = y0 + py;
  const bool valid = gx < L.width && gy < L.height;
  const bool flagged = valid && G.flags[(long long)gy * G.pitch + gx] != 0;
  if (valid && !flagged) store_px(L, gx, gy, t.raw[(py + R) * t.sw + px + R]);
  if (flagged) t.list[atomicAdd(&s_count, 1)] = threadIdx.x;
  __syncthreads();
  const int count = s_count;
  float* sagg = t.agg + threadIdx.x;
  const int stride = blockDim.x;
  const bool want_tie = L.stats != nullptr;
  int ties = 0;
  for (int k = threadIdx.x; k < count; k += blockDim.x) {
    const int id = t.list[k];
    const int qx = id % kTX, qy = id / kTX;
    uint32_t v;
    if constexpr (CRIT == kAMNFE || CRIT == kAMNFG) {
      bool tie = false;
      v = amnf_pixel<W, REG, CRIT, APX, DEG>(L, t, qx, qy, stride, tie);
      ties += tie;
    } else if constexpr (CRIT == kVMF) {
      Selection s = window_select<W, REG>(t.raw, t.sw, qx, qy, TermL2U8{}, sagg, stride, want_tie);
      v = t.raw[(qy + s.best / W) * t.sw + qx + s.best % W];
      ties += s.near_tie;
    } else if constexpr (APX == kExact) {
      Selection s =
          window_select<W, REG>(t.px, t.sw, qx, qy, TermAngleExact(L.c.a), sagg, stride, want_tie);
      v = t.raw[(qy + s.best / W) * t.sw + qx + s.best % W];
      ties += s.near_tie;
    } else {
      Selection s = window_select<W, REG>(t.px, t.sw, qx, qy, TermAngleApprox<DEG>(L.c.a, L.c.b),
                                          sagg, stride, want_tie);
      v = t.raw[(qy + s.best / W) * t.sw + qx + s.best % W];
      ties += s.near_tie;
    }
    store_px(L, x0 + qx, y0 + qy, v);
  }
  block_stats(L, valid ? 1 : 0, ties, flagged ? 1 : 0);
}

template <int W, int CRIT, int APX, int DEG>
cudaError_t launch_gated_one(const Launch& L, const GateFlags& G, int ty, int grid,
                             cudaStream_t s) {
  const size_t smem = smem_bytes(W, CRIT, ty);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(gated_kernel<W, CRIT, APX, DEG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  gated_kernel<W, CRIT, APX, DEG><<<grid, kTX * ty, smem, s>>>(L, G);
  return cudaGetLastError();
}

// AMNF per-sample approximants run as zero-padded degree 6 (bit-identical).
template <int W>
cudaError_t launch_gated_w(const Launch& L, const GateFlags& G, int crit, int apx, int degree,
                           int ty, int grid, cudaStream_t s) {
  switch (crit) {
    case kVMF: return launch_gated_one<W, kVMF, kExact, 0>(L, G, ty, grid, s);
    case kBVDF:
      if (apx == kExact) return launch_gated_one<W, kBVDF, kExact, 0>(L, G, ty, grid, s);
      switch (degree) {
        case 2: return launch_gated_one<W, kBVDF, kPoly, 2>(L, G, ty, grid, s);
        case 3: return launch_gated_one<W, kBVDF, kPoly, 3>(L, G, ty, grid, s);
        case 4: return launch_gated_one<W, kBVDF, kPoly, 4>(L, G, ty, grid, s);
        case 5: return launch_gated_one<W, kBVDF, kPoly, 5>(L, G, ty, grid, s);
        case 6: return launch_gated_one<W, kBVDF, kPoly, 6>(L, G, ty, grid, s);
        default: return cudaErrorInvalidValue;
      }
    case kAMNFE:
      if (apx == kExact) return launch_gated_one<W, kAMNFE, kExact, 0>(L, G, ty, grid, s);
      if (apx == kPoly) return launch_gated_one<W, kAMNFE, kPoly, 6>(L, G, ty, grid, s);
      return launch_gated_one<W, kAMNFE, kRational, 4>(L, G, ty, grid, s);
    case kAMNFG:
      if (apx == kExact) return launch_gated_one<W, kAMNFG, kExact, 0>(L, G, ty, grid, s);
      if (apx == kPoly) return launch_gated_one<W, kAMNFG, kPoly, 6>(L, G, ty, grid, s);
      return launch_gated_one<W, kAMNFG, kRational, 4>(L, G, ty, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace vf
