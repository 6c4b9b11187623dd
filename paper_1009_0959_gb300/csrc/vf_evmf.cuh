// vf_evmf.cuh -- the entropy vector median filter (Sec. 3.3, Eq. equ_evf) as
// a persistent kernel with a work queue.
//
// Per window the EVMF first decides the switch (mean, distances to it,
// entropy sum: O(n)) and only the switched windows need the vector median
// (O(n^2) pairs).  In the one-tile-per-CTA kernel the switched pixels of a
// tile are compacted and only that fraction of the threads runs the pair loop
// while the rest wait at the end of the tile.  Here each CTA walks a strided
// sequence of tiles and appends the window of every switched pixel (n packed
// pixels, copied from the staged tile) to a ring queue in shared memory; as
// soon as the queue holds one entry per thread, every thread takes one and
// runs the pair loop, so the O(n^2) phase always runs on full warps.  The
// queue outlives the tile it came from, so the next tile can be staged while
// entries of the previous one are still waiting.  A final partial batch
// drains the queue.
#pragma once

#include <atomic>

#include "vf_kernels.cuh"

namespace vf {

// Tile rows of the queue kernel: evmf_queue_rows (vf_internal.h); larger
// windows take 4, whose shared-memory aggregate slots and larger queue
// entries would leave one CTA per SM.

// Queue of 2 * threads entries: fewer than `threads` wait after a batch, and
// one tile adds at most `threads`.
inline size_t evmf_queue_smem_bytes(int w, int ty) {
  const size_t sw = kTX + w - 1, sh = ty + w - 1, threads = (size_t)kTX * ty;
  size_t b = sw * sh * 20;                                           // staged tile
  if (!uses_reg_path(w, kEVMF)) b += (size_t)w * w * threads * 4;   // aggregate slots
  b += 2 * threads * ((size_t)w * w * 4 + 8);                        // queue
  return b;
}

template <int W, int APX, int DEG, bool REG = uses_reg_path(W, kEVMF)>
__global__ void __launch_bounds__(256, 3) evmf_queue_kernel(const __grid_constant__ Launch L,
                                                         int ntiles) {
  constexpr int N = W * W, R = W / 2;
  pdl_begin();
  const int T = blockDim.x, TY = T / kTX, CAP = 2 * T;
  const TileSmem t = carve(W, REG, TY, T);
  // the queue starts where the one-tile kernel keeps its compaction list (an
  // 8-byte aligned offset: the tile and slot sizes are multiples of 8 bytes)
  int2* qpos = reinterpret_cast<int2*>(t.list);               // CAP output coordinates
  uint32_t* qwin = reinterpret_cast<uint32_t*>(qpos + CAP);  // CAP x N packed pixels
  __shared__ int s_tail;
  if (threadIdx.x == 0) s_tail = 0;

  const int lane = threadIdx.x & 31;
  const int px = threadIdx.x % kTX, py = threadIdx.x / kTX;
  float* sagg = t.agg + threadIdx.x;
  const bool want_tie = L.stats != nullptr;
  int head = 0;  // same value in every thread
  int pixels = 0, ties = 0, switched = 0;

  // vector median (first branch of Eq. equ_evf) of queue entry e
  auto median = [&](int e) {
    const int slot = e % CAP;
    const uint32_t* win = qwin + (size_t)slot * N;
    Selection s = window_select<W, REG>(win, W, 0, 0, TermL2U8{}, sagg, T, want_tie);
    const int2 p = qpos[slot];
    store_px(L, p.x, p.y, win[s.best]);
    ties += s.near_tie;
  };

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
    const int x0 = txi * kTX, y0 = tyi * TY;
    // the previous tile's reads of the staged pixels and the queue reads of
    // its batch end at this barrier's predecessor; staging touches only the
    // tile, the queue writes below come after the next barrier
    stage_tile<kEVMF>(L, t, x0, y0, R);
    __syncthreads();

    const int gx = x0 + px, gy = y0 + py;
    const bool valid = gx < L.width && gy < L.height;
    bool tie = false;
    const bool sw = valid && evmf_switch<W, APX, DEG>(L, t, px, py, tie);
    pixels += valid;
    ties += valid && tie;
    switched += sw;
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
      qpos[slot] = make_int2(gx, gy);
    }
    __syncthreads();
    const int tail = s_tail;
    if (tail - head >= T) {  // uniform: every thread read the same tail
      median(head + (int)threadIdx.x);
      head += T;
    }
    // s_tail is next written after the next tile's first barrier, when every
    // thread has read it; the queue slots of this batch likewise
  }
  __syncthreads();
  const int tail = s_tail;
  if ((int)threadIdx.x < tail - head) median(head + (int)threadIdx.x);
  block_stats(L, pixels, ties, switched);
}

// Persistent launch: at most as many CTAs as are resident at once, the tiles
// spread evenly over them.
template <int W, int APX, int DEG>
cudaError_t launch_evmf_queue(const Launch& L, int ty, int ntiles, cudaStream_t s) {
  // the queue kernel's own tile rows, whatever the context's per-window ones
  if (ty != evmf_queue_rows(W)) {
    ty = evmf_queue_rows(W);
    ntiles = L.tiles_x * ((L.height + ty - 1) / ty);
  }
  auto kern = evmf_queue_kernel<W, APX, DEG>;
  const int threads = kTX * ty;
  const size_t smem = evmf_queue_smem_bytes(W, ty);
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // resident CTAs per device and tile height, cached per instantiation as
  // one word (device << 40 | ty << 32 | CTAs) so concurrent callers never see
  // a torn entry
  static std::atomic<long long> cache{-1};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const long long key = ((long long)dev << 40) | ((long long)ty << 32);
  long long c = cache.load(std::memory_order_relaxed);
  if (c < 0 || (c & ~0xffffffffLL) != key) {
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    c = key | (long long)(sms * (per_sm > 0 ? per_sm : 1));
    cache.store(c, std::memory_order_relaxed);
  }
  const int ctas = (int)(c & 0xffffffffLL);
  int grid = ntiles < ctas ? ntiles : ctas;
  if (grid < 1) grid = 1;
  const int per = (ntiles + grid - 1) / grid;  // tiles per CTA
  grid = (ntiles + per - 1) / per;
  return launch_maybe_pdl(L.pdl != 0, kern, dim3(grid), dim3(threads), smem, s, L, ntiles);
}

}  // namespace vf
