// vf_gated.cuh -- the window filters restricted to the pixels a flag map
// marks (the learned gate's output); every other pixel is copied.  The flagged
// pixels of a tile are compacted in shared memory first, so the threads of a
// CTA work only on them (no divergence over copied pixels).
#pragma once

#include <algorithm>

#include "vf_kernels.cuh"

namespace vf {

struct GateFlags {
  const uint8_t* flags;  // one byte per pixel, non-zero = filter
  long long pitch;
};

template <int W, int CRIT, int APX, int DEG>
__global__ void __launch_bounds__(256) gated_kernel(const __grid_constant__ Launch L,
                                                    const GateFlags G) {
  if (L.gate_count != nullptr && *L.gate_count <= L.gate_limit) return;  // the sparse form ran
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

// Sparse form: the flagged pixels of the whole image, listed (as y * width
// + x) by the compaction kernel, which also copied every other pixel.  One
// thread per listed pixel stages its own window (borders replicated, as the
// tile kernels stage theirs) into its slice of shared memory and runs the
// per-window kernel's code on it, so a listed pixel gets exactly the
// per-window kernel's output.  Persistent CTAs; nothing to do when the list
// is longer than `limit` (the tile form then runs).
constexpr int sparse_threads(int w) { return w <= 3 ? 256 : (w == 5 ? 128 : 64); }

template <int W, int CRIT, int APX, int DEG>
__global__ void __launch_bounds__(sparse_threads(W))
    gated_sparse_kernel(const __grid_constant__ Launch L, const int* __restrict__ list,
                        const unsigned* __restrict__ count, unsigned limit) {
  constexpr int R = W / 2, N = W * W, NT = sparse_threads(W);
  constexpr bool REG = uses_reg_path(W, CRIT);
  const unsigned n = *count;
  if (n > limit) return;
  extern __shared__ __align__(16) unsigned char smem[];
  TileSmem t;  // this thread's window: W x W samples, pitch W
  t.px = reinterpret_cast<float4*>(smem) + threadIdx.x * N;
  t.raw = reinterpret_cast<uint32_t*>(smem + NT * N * 16) + threadIdx.x * N;
  t.agg = reinterpret_cast<float*>(smem + NT * N * 20);  // N slots per thread, stride NT
  t.list = nullptr;
  t.sw = W;
  t.sh = W;
  float* sagg = t.agg + threadIdx.x;
  const bool want_tie = L.stats != nullptr;
  int ties = 0;
  for (unsigned k = blockIdx.x * NT + threadIdx.x; k < n; k += gridDim.x * NT) {
    const int id = list[k];
    const int y = id / L.width, x = id - y * L.width;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int gy = min(max(y + i / W - R, 0), L.height - 1);
      const int gx = min(max(x + i % W - R, 0), L.width - 1);
      const uint32_t v = load_px(L, gx, gy);
      t.raw[i] = v;
      if constexpr (CRIT != kVMF) t.px[i] = stage_cell<CRIT>(v);
    }
    uint32_t v;
    if constexpr (CRIT == kAMNFE || CRIT == kAMNFG) {
      bool tie = false;
      v = amnf_pixel<W, REG, CRIT, APX, DEG>(L, t, 0, 0, NT, tie);
      ties += tie;
    } else if constexpr (CRIT == kVMF) {
      Selection s = window_select<W, REG>(t.raw, W, 0, 0, TermL2U8{}, sagg, NT, want_tie);
      v = t.raw[s.best];
      ties += s.near_tie;
    } else if constexpr (APX == kExact) {
      Selection s =
          window_select<W, REG>(t.px, W, 0, 0, TermAngleExact(L.c.a), sagg, NT, want_tie);
      v = t.raw[s.best];
      ties += s.near_tie;
    } else {
      Selection s = window_select<W, REG>(t.px, W, 0, 0, TermAngleApprox<DEG>(L.c.a, L.c.b),
                                          sagg, NT, want_tie);
      v = t.raw[s.best];
      ties += s.near_tie;
    }
    store_px(L, x, y, v);
  }
  // every pixel of the image and the flagged ones, counted once
  const bool first = blockIdx.x == 0 && threadIdx.x == 0;
  block_stats(L, first ? L.width * L.height : 0, ties, first ? (int)n : 0);
}

template <int W, int CRIT, int APX, int DEG>
cudaError_t launch_sparse_one(const Launch& L, const int* list, const unsigned* count,
                              unsigned limit, int sms, cudaStream_t s) {
  constexpr int NT = sparse_threads(W), N = W * W;
  const size_t smem = (size_t)NT * N * 24;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(gated_sparse_kernel<W, CRIT, APX, DEG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, gated_sparse_kernel<W, CRIT, APX, DEG>, NT, smem);
  if (e != cudaSuccess) return e;
  gated_sparse_kernel<W, CRIT, APX, DEG>
      <<<std::max(per_sm, 1) * sms, NT, smem, s>>>(L, list, count, limit);
  return cudaGetLastError();
}

// AMNF per-sample approximants run as zero-padded degree 6 (bit-identical).
template <int W>
cudaError_t launch_sparse_w(const Launch& L, const int* list, const unsigned* count,
                            unsigned limit, int sms, int crit, int apx, int degree,
                            cudaStream_t s) {
  switch (crit) {
    case kVMF: return launch_sparse_one<W, kVMF, kExact, 0>(L, list, count, limit, sms, s);
    case kBVDF:
      if (apx == kExact) return launch_sparse_one<W, kBVDF, kExact, 0>(L, list, count, limit, sms, s);
      switch (degree) {
        case 2: return launch_sparse_one<W, kBVDF, kPoly, 2>(L, list, count, limit, sms, s);
        case 3: return launch_sparse_one<W, kBVDF, kPoly, 3>(L, list, count, limit, sms, s);
        case 4: return launch_sparse_one<W, kBVDF, kPoly, 4>(L, list, count, limit, sms, s);
        case 5: return launch_sparse_one<W, kBVDF, kPoly, 5>(L, list, count, limit, sms, s);
        case 6: return launch_sparse_one<W, kBVDF, kPoly, 6>(L, list, count, limit, sms, s);
        default: return cudaErrorInvalidValue;
      }
    case kAMNFE:
      if (apx == kExact) return launch_sparse_one<W, kAMNFE, kExact, 0>(L, list, count, limit, sms, s);
      if (apx == kPoly) return launch_sparse_one<W, kAMNFE, kPoly, 6>(L, list, count, limit, sms, s);
      return launch_sparse_one<W, kAMNFE, kRational, 4>(L, list, count, limit, sms, s);
    case kAMNFG:
      if (apx == kExact) return launch_sparse_one<W, kAMNFG, kExact, 0>(L, list, count, limit, sms, s);
      if (apx == kPoly) return launch_sparse_one<W, kAMNFG, kPoly, 6>(L, list, count, limit, sms, s);
      return launch_sparse_one<W, kAMNFG, kRational, 4>(L, list, count, limit, sms, s);
    default: return cudaErrorInvalidValue;
  }
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
