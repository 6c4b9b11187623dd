// vf_batch_class.cuh -- class kernels of the batched form: one persistent
// kernel per image class (window x criterion x approximation), each with the
// tile shape, block size and shared memory of that class's single-image
// kernel, pulling the tiles of every image of its class from its own queue.
//
// The single persistent kernel of vf_batch.cu hosts every class in one block
// shape, so its register count, shared memory and tile rows are the maximum
// over all classes (and the tall pair-reuse tiles of BVDF, which need 864
// threads and most of the shared memory, cannot run in it at all).  Here each
// class runs the body its single-image launch runs -- two windows per thread
// for VMF and AMNF, the tall pair-reuse tiles for BVDF, the per-window tiles
// with compaction for EVMF -- and the class kernels of one batch run
// concurrently (one CUDA graph with a branch per class), so the tail of one
// class overlaps the next.
#pragma once

#include "vf_evmf.cuh"
#include "vf_kernels.cuh"
#include "vf_reuse.cuh"

namespace vf {

struct BatchImage {
  Launch L;
  int cls;
  int two;  // single kernel: 1 = two windows per thread (tiles of 32 x 2TY outputs)
};

// Body of a class: 0 two windows per thread (VMF, AMNFE, AMNFG), 1 the tall
// pair-reuse tiles (BVDF), 2 per-window tiles with compaction (EVMF 3 x 3
// and 7 x 7), 3 the EVMF work queue (EVMF 5 x 5), as the single-image
// launches choose them.
constexpr int class_body(int w, int crit) {
  return crit == kBVDF ? 1 : (crit == kEVMF ? (w == 5 ? 3 : 2) : 0);
}
// Thread rows of the two-window and per-window bodies (32 x 4 threads).
constexpr int kClassTY = 4;
// Output rows of one tile of a class.
constexpr int class_rows(int w, int crit) {
  return class_body(w, crit) == 1   ? reuse_tile_rows(w, kBVDF)
         : class_body(w, crit) == 0 ? 2 * kClassTY
         : class_body(w, crit) == 3 ? evmf_queue_rows(w)
                                    : kClassTY;
}
constexpr int class_threads(int w, int crit) {
  return class_body(w, crit) == 1   ? reuse_threads(w, reuse_tile_rows(w, kBVDF))
         : class_body(w, crit) == 3 ? kTX * evmf_queue_rows(w)
                                    : kTX * kClassTY;
}
inline size_t class_kernel_smem(int w, int crit) {
  switch (class_body(w, crit)) {
    case 0: return smem_bytes(w, crit, 2 * kClassTY);
    case 1: return reuse_any_smem_bytes(w, reuse_tile_rows(w, kBVDF));
    case 3: return evmf_queue_smem_bytes(w, evmf_queue_rows(w));
    default: return smem_bytes(w, crit, kClassTY);
  }
}

// Output pixel reference of a queued window: its byte address with the store
// form in bits 62-63 (0 one 32-bit store, 1 three bytes, 2 four bytes), so
// that a queue entry outlives the tile (and the image) it came from.
__device__ __forceinline__ unsigned long long out_ref(const Launch& L, int gx, int gy) {
  const uint8_t* p = L.out + (long long)gy * L.out_pitch + (long long)gx * L.channels;
  const unsigned long long form = L.vec4_out ? 0ull : (L.channels == 4 ? 2ull : 1ull);
  return reinterpret_cast<unsigned long long>(p) | (form << 62);
}
__device__ __forceinline__ void store_ref(unsigned long long r, uint32_t v) {
  uint8_t* p = reinterpret_cast<uint8_t*>(r & ((1ull << 62) - 1ull));
  const unsigned form = (unsigned)(r >> 62);
  if (form == 0) {
    *reinterpret_cast<uint32_t*>(p) = v;
    return;
  }
  p[0] = (uint8_t)v;
  p[1] = (uint8_t)(v >> 8);
  p[2] = (uint8_t)(v >> 16);
  if (form == 2) p[3] = (uint8_t)(v >> 24);
}

// The EVMF work queue (evmf_queue_kernel, vf_evmf.cuh) over the tiles of
// every image of the class: each tile comes from the class counter (its
// image's descriptor staged in shared memory), and a queued window carries
// its output address instead of coordinates, so windows of different images
// share the queue and its full-warp batches.
template <int W, int APX, int DEG, bool REG = uses_reg_path(W, kEVMF)>
__global__ void __launch_bounds__(256, 3)
    evmf_class_kernel(const BatchImage* __restrict__ imgs, const int* __restrict__ begin,
                      int count, unsigned int* counter) {
  constexpr int N = W * W, R = W / 2;
  const int T = blockDim.x, TY = T / kTX, CAP = 2 * T;
  const TileSmem t = carve(W, REG, TY, T);
  unsigned long long* qdst = reinterpret_cast<unsigned long long*>(t.list);  // CAP outputs
  uint32_t* qwin = reinterpret_cast<uint32_t*>(qdst + CAP);                  // CAP x N pixels
  __shared__ int s_tail, s_item;
  __shared__ Launch s_L;
  if (threadIdx.x == 0) s_tail = 0;
  const int lane = threadIdx.x & 31;
  const int px = threadIdx.x % kTX, py = threadIdx.x / kTX;
  float* sagg = t.agg + threadIdx.x;
  const int total = begin[count];
  int head = 0;  // same value in every thread

  auto median = [&](int e) {
    const int slot = e % CAP;
    const uint32_t* win = qwin + (size_t)slot * N;
    const Selection s = window_select<W, REG>(win, W, 0, 0, TermL2U8{}, sagg, T, false);
    store_ref(qdst[slot], win[s.best]);
  };

  for (;;) {
    __syncthreads();  // staged pixels, s_L and s_item of the previous tile are done
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    int lo = 0, hi = count - 1;  // largest i with begin[i] <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (begin[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const int tile = item - begin[lo];
    if (threadIdx.x < 32) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&imgs[lo].L);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&s_L);
      for (int k = threadIdx.x; k < (int)(sizeof(Launch) / 4); k += 32) dst[k] = src[k];
    }
    __syncthreads();
    const Launch& L = s_L;
    const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
    const int x0 = txi * kTX, y0 = tyi * TY;
    stage_tile<kEVMF>(L, t, x0, y0, R);
    __syncthreads();
    const int gx = x0 + px, gy = y0 + py;
    const bool valid = gx < L.width && gy < L.height;
    bool tie = false;
    const bool sw = valid && evmf_switch<W, APX, DEG>(L, t, px, py, tie);
    if (valid && !sw) store_px(L, gx, gy, t.raw[(py + R) * t.sw + px + R]);
    // warp-aggregated append: consecutive slots for a warp's switched pixels
    const unsigned m = __ballot_sync(0xffffffffu, sw);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(&s_tail, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (sw) {
      const int slot = (base + __popc(m & ((1u << lane) - 1u))) % CAP;
      uint32_t* dst = qwin + (size_t)slot * N;
#pragma unroll
      for (int a = 0; a < W; ++a)
#pragma unroll
        for (int i = 0; i < W; ++i) dst[a * W + i] = t.raw[(py + a) * t.sw + px + i];
      qdst[slot] = out_ref(L, gx, gy);
    }
    __syncthreads();
    const int tail = s_tail;
    if (tail - head >= T) {  // uniform: every thread read the same tail
      median(head + (int)threadIdx.x);
      head += T;
    }
  }
  __syncthreads();
  const int tail = s_tail;
  if ((int)threadIdx.x < tail - head) median(head + (int)threadIdx.x);
}

// begin[i] = first tile of the class's image i, begin[count] = its tiles.
template <int W, int CRIT, int APX, int DEG>
__global__ void __launch_bounds__(class_threads(W, CRIT))
    class_kernel(const BatchImage* __restrict__ imgs, const int* __restrict__ begin, int count,
                 unsigned int* counter) {
  __shared__ int s_item;
  __shared__ Launch s_L;  // the current tile's image
  const int total = begin[count];
  for (;;) {
    __syncthreads();  // the previous tile is done with shared memory and s_item
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= total) return;
    int lo = 0, hi = count - 1;  // largest i with begin[i] <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (begin[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const int tile = item - begin[lo];
    static_assert(sizeof(Launch) % 4 == 0, "descriptor is copied as words");
    if (threadIdx.x < 32) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&imgs[lo].L);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&s_L);
      for (int k = threadIdx.x; k < (int)(sizeof(Launch) / 4); k += 32) dst[k] = src[k];
    }
    __syncthreads();
    if constexpr (class_body(W, CRIT) == 0) {
      process_tile2<W, CRIT, APX, DEG>(s_L, tile);
    } else if constexpr (class_body(W, CRIT) == 1) {
      constexpr int RTY = reuse_tile_rows(W, kBVDF);
      reuse_any_tile<W, kBVDF, APX, DEG, RTY, reuse_threads(W, RTY)>(s_L, tile);
    } else {
      process_tile<W, CRIT, APX, DEG>(s_L, tile);
    }
  }
}

// Launches the class kernel of one window, criterion and approximation on
// `s`: as many CTAs as are resident at once on the device, or `tiles` when
// the class has fewer tiles.
template <int W, int CRIT, int APX, int DEG>
cudaError_t launch_class_one(const BatchImage* imgs, const int* begin, int count,
                             unsigned int* counter, int tiles, cudaStream_t s) {
  void (*kern)(const BatchImage*, const int*, int, unsigned int*);
  if constexpr (class_body(W, CRIT) == 3) kern = evmf_class_kernel<W, APX, DEG>;
  else kern = class_kernel<W, CRIT, APX, DEG>;
  const size_t smem = class_kernel_smem(W, CRIT);
  const int threads = class_threads(W, CRIT);
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  int grid = sms * (per_sm > 0 ? per_sm : 1);
  if (tiles < grid) grid = tiles;
  if (grid < 1) grid = 1;
  kern<<<grid, threads, smem, s>>>(imgs, begin, count, counter);
  return cudaGetLastError();
}

// exact, polynomial (degree 6, zero-padded) or rational (4,4) for one window
// and criterion
template <int W, int CRIT>
cudaError_t launch_class_apx(int apx, const BatchImage* imgs, const int* begin, int count,
                             unsigned int* counter, int tiles, cudaStream_t s) {
  if (apx == kExact) return launch_class_one<W, CRIT, kExact, 0>(imgs, begin, count, counter, tiles, s);
  if (apx == kPoly) return launch_class_one<W, CRIT, kPoly, 6>(imgs, begin, count, counter, tiles, s);
  if constexpr (CRIT != kBVDF) {
    if (apx == kRational)
      return launch_class_one<W, CRIT, kRational, 4>(imgs, begin, count, counter, tiles, s);
  }
  return cudaErrorInvalidValue;
}

template <int W>
cudaError_t launch_class_window(int crit, int apx, const BatchImage* imgs, const int* begin,
                                int count, unsigned int* counter, int tiles, cudaStream_t s) {
  switch (crit) {
    case kVMF: return launch_class_one<W, kVMF, kExact, 0>(imgs, begin, count, counter, tiles, s);
    case kBVDF: return launch_class_apx<W, kBVDF>(apx, imgs, begin, count, counter, tiles, s);
    case kAMNFE: return launch_class_apx<W, kAMNFE>(apx, imgs, begin, count, counter, tiles, s);
    case kAMNFG: return launch_class_apx<W, kAMNFG>(apx, imgs, begin, count, counter, tiles, s);
    case kEVMF: return launch_class_apx<W, kEVMF>(apx, imgs, begin, count, counter, tiles, s);
    default: return cudaErrorInvalidValue;
  }
}

// One translation unit per window (vf_bc_w<w>.cu).
cudaError_t launch_class_w3(int crit, int apx, const BatchImage* imgs, const int* begin, int count,
                            unsigned int* counter, int tiles, cudaStream_t s);
cudaError_t launch_class_w5(int crit, int apx, const BatchImage* imgs, const int* begin, int count,
                            unsigned int* counter, int tiles, cudaStream_t s);
cudaError_t launch_class_w7(int crit, int apx, const BatchImage* imgs, const int* begin, int count,
                            unsigned int* counter, int tiles, cudaStream_t s);

}  // namespace vf
