// vf_batch.cu -- many images of uneven sizes, mixed windows and criteria in
// one persistent launch (and as a CUDA graph), with an autotuner for the tile
// shape and the number of resident CTAs.
//
// The host flattens the batch into one queue of 32 x TY output tiles, images
// ordered by decreasing estimated cost per tile (longest-processing-time
// first, so the tail of the queue holds the cheap tiles).  A grid of
// (SMs x CTAs per SM) CTAs pulls tile indices from a global counter with one
// atomicAdd per tile; no CTA ever waits on another.  A tile is mapped to its
// image by binary search over the images' first tile indices, then run by the
// same per-tile body as the single-image kernel (vf_kernels.cuh), selected by
// the image's class (window x criterion x approximation); BVDF tiles run the
// pair-reuse body (vf_reuse.cuh) when the tiles are 32 x 8.  Polynomials run
// as degree 6 with zero-padded coefficients (fma(0, z, c) = c exactly, so the
// result is bit-identical to the degree-specific kernel).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "vf_batch_class.cuh"
#include "vf_kernels.cuh"
#include "vf_reuse.cuh"

namespace vf {

// Kernel classes: window (3, 5, 7) x 12 criterion/approximation pairs.
constexpr int kClassesPerWindow = 12;
__host__ __device__ constexpr int class_of(int w, int crit, int apx) {
  int k = 0;
  switch (crit) {
    case kVMF: k = 0; break;
    case kBVDF: k = 1 + (apx != kExact); break;
    case kAMNFE: k = 3 + apx; break;
    case kAMNFG: k = 6 + apx; break;
    default: k = 9 + apx; break;
  }
  return (w == 3 ? 0 : (w == 5 ? 1 : 2)) * kClassesPerWindow + k;
}

// Inside the batch kernel 3 x 3 keeps its aggregates in registers, and so
// does the 5 x 5 AMNF (its integer city-block path needs about 64
// registers); the other 5 x 5 register bodies (about 127 registers) would
// force spills into every class, since the kernel's register budget is that
// of its largest body.
constexpr bool batch_reg(int w, int crit) {
  return w == 3 || (w == 5 && (crit == kAMNFE || crit == kAMNFG));
}

// Class decoding (inverse of class_of for window and criterion).
__host__ __device__ constexpr int class_window(int cls) { return 3 + 2 * (cls / kClassesPerWindow); }
__host__ __device__ constexpr int class_crit(int cls) {
  const int k = cls % kClassesPerWindow;
  return k == 0 ? kVMF : (k <= 2 ? kBVDF : (k <= 5 ? kAMNFE : (k <= 8 ? kAMNFG : kEVMF)));
}

// AMNF with w <= 5 and VMF 3 x 3 run the two-windows-per-thread body: their
// tiles are 32 x 2TY, the others 32 x TY.  (The 5 x 5 VMF two-window body
// needs about 128 registers, which would spill in the shared kernel.)
__host__ __device__ constexpr int batch_rows_per_thread(int w, int crit) {
  return (outputs_per_thread(w, crit) == 2 && w <= 5 && !(crit == kVMF && w == 5)) ? 2 : 1;
}

// The in-register two-window body exists for VMF and AMNF with w <= 5.
__host__ __device__ constexpr bool batch_two_available(int w, int crit) {
  return outputs_per_thread(w, crit) == 2 && w <= 5;
}

// Whether an image runs two windows per thread under the batch's
// pixels-per-thread setting: 0 the per-class default above, 1 never, 2
// wherever the body exists.
__host__ __device__ constexpr int batch_two(int ppt, int w, int crit) {
  return !batch_two_available(w, crit) ? 0
         : ppt == 0                     ? (batch_rows_per_thread(w, crit) == 2 ? 1 : 0)
                                        : (ppt == 2 ? 1 : 0);
}

template <int W, int CRIT, int APX, int DEG, bool REG>
__device__ __forceinline__ void run_one(const Launch& L, int tile, int two) {
  if constexpr (batch_two_available(W, CRIT)) {
    if (two) {
      process_tile2<W, CRIT, APX, DEG>(L, tile);
      return;
    }
  }
  process_tile<W, CRIT, APX, DEG, REG>(L, tile);
}

template <int W>
__device__ __forceinline__ void run_class(int k, const Launch& L, int tile, int two) {
  constexpr bool RG = batch_reg(W, kVMF);
  constexpr bool RA = batch_reg(W, kAMNFE);
  switch (k) {
    case 0: run_one<W, kVMF, kExact, 0, RG>(L, tile, two); break;
    // BVDF: with 32 x 8 tiles (256 threads) the pair-reuse body, whose tile
    // grid is the same; otherwise the per-window body
    case 1:
      if (blockDim.x == kRTX * kRTY) reuse_any_tile<W, kBVDF, kExact, 0>(L, tile);
      else process_tile<W, kBVDF, kExact, 0, RG>(L, tile);
      break;
    case 2:
      if (blockDim.x == kRTX * kRTY) reuse_any_tile<W, kBVDF, kPoly, 6>(L, tile);
      else process_tile<W, kBVDF, kPoly, 6, RG>(L, tile);
      break;
    case 3: run_one<W, kAMNFE, kExact, 0, RA>(L, tile, two); break;
    case 4: run_one<W, kAMNFE, kPoly, 6, RA>(L, tile, two); break;
    case 5: run_one<W, kAMNFE, kRational, 4, RA>(L, tile, two); break;
    case 6: run_one<W, kAMNFG, kExact, 0, RA>(L, tile, two); break;
    case 7: run_one<W, kAMNFG, kPoly, 6, RA>(L, tile, two); break;
    case 8: run_one<W, kAMNFG, kRational, 4, RA>(L, tile, two); break;
    case 9: process_tile<W, kEVMF, kExact, 0, RG>(L, tile); break;
    case 10: process_tile<W, kEVMF, kPoly, 6, RG>(L, tile); break;
    default: process_tile<W, kEVMF, kRational, 4, RG>(L, tile); break;
  }
}

// begin[i] = first tile of image i in the queue, begin[count] = total tiles.
__global__ void __launch_bounds__(256, 2) batch_kernel(const BatchImage* __restrict__ imgs,
                                                       const int* __restrict__ begin, int count,
                                                       unsigned int* counter) {
  __shared__ int s_item;
  __shared__ BatchImage s_img;  // the current tile's image descriptor
  const int total = begin[count];
  for (;;) {
    __syncthreads();  // the previous tile is done with shared memory and s_item
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= total) return;
    int lo = 0, hi = count - 1;  // largest i with begin[i] <= item
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (begin[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const int tile = item - begin[lo];
    // stage the descriptor once per tile (word copy by the first warp)
    static_assert(sizeof(BatchImage) % 4 == 0, "descriptor is copied as words");
    if (threadIdx.x < 32) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(imgs + lo);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&s_img);
      for (int k = threadIdx.x; k < (int)(sizeof(BatchImage) / 4); k += 32) dst[k] = src[k];
    }
    __syncthreads();
    const Launch& L = s_img.L;
    const int cls = s_img.cls, two = s_img.two;
    const int wi = cls / kClassesPerWindow, k = cls - wi * kClassesPerWindow;
    if (wi == 0) run_class<3>(k, L, tile, two);
    else if (wi == 1) run_class<5>(k, L, tile, two);
    else run_class<7>(k, L, tile, two);
  }
}

// Relative cost of one output pixel per class (pairs x term cost), used only
// to order the queue.
static double pixel_cost(const LaunchClass& c) {
  const double n = (double)c.w * c.w, pairs = n * (n - 1) / 2;
  double term = 1.0;
  switch (c.crit) {
    case kVMF: term = 1.0; break;
    case kBVDF: term = c.apx == kExact ? 7.0 : 3.5; break;
    case kAMNFE:
    case kAMNFG: term = 1.0; break;
    default: term = 0.5; break;
  }
  return pairs * term;
}

}  // namespace vf

using namespace vf;

// One class of the class-kernel form: images [first, first + count) of the
// class queue, its prefix array at begin_off, its counter, its tiles.
struct BatchClass {
  int w, crit, apx;
  int first, count, begin_off, tiles;
  double cost;    // estimated work (tiles x pixels x cost per pixel)
  int per_image;  // 1: the class's images go as single-image launches instead
};

constexpr int kBatchBranches = 4;  // concurrent branches of the class-kernel form

struct vf_batch {
  vf_ctx* ctx = nullptr;
  int mode = VF_BATCH_ONE_KERNEL;
  // class-kernel form: descriptors grouped by class, prefix arrays, counters
  std::vector<BatchClass> classes;
  BatchImage* d_cimgs = nullptr;
  int* d_cbegin = nullptr;
  unsigned int* d_ccounters = nullptr;
  cudaStream_t branch[kBatchBranches] = {};
  cudaEvent_t fork = nullptr, join[kBatchBranches] = {};
  int device = 0, sms = 0;
  std::vector<BatchImage> host;  // queue order
  std::vector<LaunchClass> host_cls;  // the images' kernel classes, queue order
  std::vector<int> cls_img;           // class-kernel form: host index of each grouped image
  std::vector<double> cost;
  BatchImage* d_imgs = nullptr;
  int* d_begin = nullptr;
  unsigned int* d_counter = nullptr;
  int count = 0;
  int ty = 4, ctas_per_sm = 0;  // 0: occupancy maximum
  int ppt = 0;                  // pixels per thread: 0 per-class default, 1, 2
  size_t smem = 0;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

// Shared memory of one class's body with CTAs of 32 x ty threads.
size_t class_smem(int w, int crit, int ty, int two) {
  if (two) return smem_bytes(w, crit, 2 * ty, true);
  size_t m = smem_bytes(w, crit, ty, batch_reg(w, crit));
  if (crit == kBVDF && kTX * ty == kRTX * kRTY) m = std::max(m, reuse_any_smem_bytes(w));
  return m;
}

size_t batch_smem(const vf_batch* b, int ty) {
  size_t m = 0;
  for (const BatchImage& im : b->host) {
    const int w = class_window(im.cls), crit = class_crit(im.cls);
    m = std::max(m, class_smem(w, crit, ty, batch_two(b->ppt, w, crit)));
  }
  return m;
}

// Tile counts for TY = ty; uploads descriptors and the prefix array.
vf_status upload(vf_batch* b, int ty) {
  std::vector<int> begin(b->count + 1, 0);
  for (int i = 0; i < b->count; ++i) {
    Launch& L = b->host[i].L;
    const int cls = b->host[i].cls;
    b->host[i].two = batch_two(b->ppt, class_window(cls), class_crit(cls));
    const int rows = ty * (b->host[i].two ? 2 : 1);
    L.tiles_x = (L.width + kTX - 1) / kTX;
    long long tiles = (long long)L.tiles_x * ((L.height + rows - 1) / rows);
    long long next = (long long)begin[i] + tiles;
    if (next > 0x7fffffffLL) return set_error(b->ctx, VF_ERR_UNSUPPORTED, "batch too large");
    begin[i + 1] = (int)next;
  }
  cudaError_t e = cudaMemcpy(b->d_imgs, b->host.data(), sizeof(BatchImage) * b->count,
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_begin, begin.data(), sizeof(int) * (b->count + 1), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return set_error(b->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  b->ty = ty;
  b->smem = batch_smem(b, ty);
  return VF_OK;
}

vf_status drop_graph(vf_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  return VF_OK;
}

int resident_ctas(const vf_batch* b, int ty) {
  int blocks = 0;
  const size_t smem = batch_smem(b, ty);
  // the occupancy query counts a dynamic size above 48 KB only once the
  // kernel has been allowed that much
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, batch_kernel, kTX * ty, smem) !=
      cudaSuccess)
    return 1;
  return std::max(blocks, 1);
}

// Class-kernel form: group the images by class (window x criterion x
// approximation), each class's images in the queue's cost order; tile counts
// with the class's own tile rows.  Uploads the grouped descriptors and prefix
// arrays (once, at creation).
vf_status upload_classes(vf_batch* b) {
  std::vector<int> order(b->count);
  for (int i = 0; i < b->count; ++i) order[i] = i;
  b->cls_img.clear();
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->host[x].cls < b->host[y].cls; });
  std::vector<BatchImage> imgs;
  std::vector<int> begin;
  b->classes.clear();
  for (int k = 0; k < b->count;) {
    const int cls = b->host[order[k]].cls;
    BatchClass c{};
    c.w = class_window(cls);
    c.crit = class_crit(cls);
    const int kk = cls % kClassesPerWindow;
    c.apx = c.crit == kVMF ? kExact
            : c.crit == kBVDF ? (kk == 1 ? kExact : kPoly)
                              : (kk - (c.crit == kAMNFE ? 3 : (c.crit == kAMNFG ? 6 : 9)));
    c.first = (int)imgs.size();
    c.begin_off = (int)begin.size();
    const int rows = class_rows(c.w, c.crit);
    long long tiles = 0;
    double px = 0.0;
    for (; k < b->count && b->host[order[k]].cls == cls; ++k) {
      BatchImage im = b->host[order[k]];
      b->cls_img.push_back(order[k]);
      im.L.tiles_x = (im.L.width + kTX - 1) / kTX;
      begin.push_back((int)tiles);
      tiles += (long long)im.L.tiles_x * ((im.L.height + rows - 1) / rows);
      if (tiles > 0x7fffffffLL) return set_error(b->ctx, VF_ERR_UNSUPPORTED, "batch too large");
      px += (double)im.L.width * im.L.height;
      imgs.push_back(im);
    }
    begin.push_back((int)tiles);
    c.count = (int)imgs.size() - c.first;
    c.tiles = (int)tiles;
    LaunchClass lc{c.crit, c.w, c.apx, 0, 0};
    c.cost = px * pixel_cost(lc);
    // BVDF keeps one launch per image by default: its tall tiles take a whole
    // SM each, and the single-image kernel reads the approximant as
    // constant-bank operands where the class kernel reads the staged
    // descriptor (vf_batch_autotune decides per class by timing)
    c.per_image = c.crit == kBVDF;
    b->classes.push_back(c);
  }
  // costliest classes first: their kernels start first, the cheap ones fill
  // the tail
  std::stable_sort(b->classes.begin(), b->classes.end(),
                   [](const BatchClass& x, const BatchClass& y) { return x.cost > y.cost; });
  cudaError_t e = device_alloc(&b->d_cimgs, sizeof(BatchImage) * imgs.size());
  if (e == cudaSuccess) e = device_alloc(&b->d_cbegin, sizeof(int) * begin.size());
  if (e == cudaSuccess)
    e = device_alloc(&b->d_ccounters, sizeof(unsigned int) * b->classes.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_cimgs, imgs.data(), sizeof(BatchImage) * imgs.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_cbegin, begin.data(), sizeof(int) * begin.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < kBatchBranches && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(b->ctx, e == cudaErrorMemoryAllocation ? VF_ERR_OOM : VF_ERR_CUDA,
                     cudaGetErrorString(e));
  }
  return VF_OK;
}

// Class-kernel form: reset the counters on s, fork the branches from s, the
// class kernels on the branches (class i on branch i mod kBatchBranches, in
// cost order), join them back into s.
// One class on stream bs: its class kernel (its counter reset first), or one
// single-image launch per image.
cudaError_t enqueue_one_class(vf_batch* b, size_t i, cudaStream_t bs) {
  const BatchClass& c = b->classes[i];
  if (c.per_image) {
    for (int k = 0; k < c.count; ++k) {
      const int h = b->cls_img[c.first + k];
      if (launch_single(b->ctx, b->host[h].L, b->host_cls[h], bs) != VF_OK)
        return cudaErrorLaunchFailure;
    }
    return cudaSuccess;
  }
  const BatchImage* imgs = b->d_cimgs + c.first;
  const int* begin = b->d_cbegin + c.begin_off;
  unsigned int* counter = b->d_ccounters + i;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), bs);
  if (e != cudaSuccess) return e;
  return c.w == 3   ? launch_class_w3(c.crit, c.apx, imgs, begin, c.count, counter, c.tiles, bs)
         : c.w == 5 ? launch_class_w5(c.crit, c.apx, imgs, begin, c.count, counter, c.tiles, bs)
                    : launch_class_w7(c.crit, c.apx, imgs, begin, c.count, counter, c.tiles, bs);
}

vf_status enqueue_classes(vf_batch* b, cudaStream_t s) {
  const int nb = std::min<int>(kBatchBranches, (int)b->classes.size());
  cudaError_t e = cudaEventRecord(b->fork, s);
  for (int i = 0; i < nb && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
  for (size_t i = 0; i < b->classes.size() && e == cudaSuccess; ++i)
    e = enqueue_one_class(b, i, b->branch[i % nb]);
  for (int i = 0; i < nb && e == cudaSuccess; ++i) {
    e = cudaEventRecord(b->join[i], b->branch[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join[i], 0);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(b->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  }
  return VF_OK;
}

vf_status enqueue(vf_batch* b, cudaStream_t s) {
  if (b->mode == VF_BATCH_CLASS_KERNELS) return enqueue_classes(b, s);
  const int threads = kTX * b->ty;
  int per_sm = b->ctas_per_sm > 0 ? b->ctas_per_sm : resident_ctas(b, b->ty);
  const int grid = b->sms * per_sm;
  if (b->smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)b->smem);
    if (e != cudaSuccess) return set_error(b->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return set_error(b->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  batch_kernel<<<grid, threads, b->smem, s>>>(b->d_imgs, b->d_begin, b->count, b->d_counter);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(b->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  return VF_OK;
}

}  // namespace

extern "C" {

vf_status vf_batch_create(vf_ctx* ctx, const vf_image_desc* descs, int count, vf_batch** out) {
  if (!ctx) return VF_ERR_ARG;
  if (!descs || !out || count < 1) return set_error(ctx, VF_ERR_ARG, "empty batch");
  *out = nullptr;
  vf_batch* b = alloc_refused() ? nullptr : new (std::nothrow) vf_batch();
  if (!b) return VF_ERR_OOM;
  b->ctx = ctx;
  b->count = count;
  std::vector<std::pair<double, int>> order;
  std::vector<BatchImage> imgs(count);
  std::vector<LaunchClass> lcls(count);
  for (int i = 0; i < count; ++i) {
    const vf_image_desc& d = descs[i];
    LaunchClass c;
    vf_status st = prepare_launch(ctx, d.d_in, d.d_out, d.height, d.width, d.channels,
                                  d.in_pitch, d.out_pitch, &d.params, nullptr, &imgs[i].L, &c);
    if (st == VF_OK && c.precision != VF_FP32)
      st = set_error(ctx, VF_ERR_UNSUPPORTED, "the batched form runs in FP32 only");
    if (st == VF_OK && c.crit == kEVBDF)
      st = set_error(ctx, VF_ERR_UNSUPPORTED, "EVBDF runs through vf_filter only");
    if (st != VF_OK) {
      delete b;
      return st;
    }
    imgs[i].cls = class_of(c.w, c.crit, c.apx);
    lcls[i] = c;
    order.push_back({-pixel_cost(c), i});
  }
  std::stable_sort(order.begin(), order.end());
  for (auto& o : order) {
    b->host.push_back(imgs[o.second]);
    b->host_cls.push_back(lcls[o.second]);
  }
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) e = device_alloc(&b->d_imgs, sizeof(BatchImage) * count);
  if (e == cudaSuccess) e = device_alloc(&b->d_begin, sizeof(int) * (count + 1));
  if (e == cudaSuccess) e = device_alloc(&b->d_counter, sizeof(unsigned int));
  if (e != cudaSuccess) {
    vf_batch_destroy(b);
    cudaGetLastError();
    return set_error(ctx, e == cudaErrorMemoryAllocation ? VF_ERR_OOM : VF_ERR_CUDA,
                     cudaGetErrorString(e));
  }
  vf_status st = upload(b, 4);
  if (st == VF_OK) st = upload_classes(b);
  if (st != VF_OK) {
    vf_batch_destroy(b);
    return st;
  }
  *out = b;
  return VF_OK;
}

vf_status vf_batch_launch(vf_batch* b, void* stream) {
  if (!b) return VF_ERR_ARG;
  return enqueue(b, (cudaStream_t)stream);
}

vf_status vf_batch_graph_launch(vf_batch* b, void* stream) {
  if (!b) return VF_ERR_ARG;
  cudaError_t e = cudaSuccess;
  if (!b->exec) {
    if (!b->cap) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return set_error(b->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
    vf_status st = enqueue(b, b->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (st != VF_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e == cudaSuccess) {
      b->graph = g;
      e = cudaGraphInstantiate(&b->exec, g, 0);
    }
    if (e != cudaSuccess) {
      drop_graph(b);
      return set_error(b->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(b->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  return VF_OK;
}

vf_status vf_batch_autotune(vf_batch* b, void* stream, int* tile_rows, int* ctas_per_sm,
                            float* best_ms) {
  if (!b) return VF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return set_error(b->ctx, VF_ERR_CUDA, "event creation failed");
  }
  float best = 1e30f;
  int best_ty = b->ty, best_ctas = b->ctas_per_sm, best_ppt = b->ppt;
  vf_status st = VF_OK;
  const int tys[3] = {2, 4, 8};
  for (int pp = 0; pp < 9 && st == VF_OK; ++pp) {
    const int ti = pp % 3;
    b->ppt = pp / 3;  // pixels per thread: class default, 1, 2
    st = upload(b, tys[ti]);
    if (st != VF_OK) break;
    const int maxc = resident_ctas(b, tys[ti]);
    for (int c = 1; c <= maxc && st == VF_OK; ++c) {
      b->ctas_per_sm = c;
      st = enqueue(b, s);  // warm-up
      float ms_min = 1e30f;
      for (int r = 0; r < 3 && st == VF_OK; ++r) {
        cudaEventRecord(e0, s);
        st = enqueue(b, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = set_error(b->ctx, VF_ERR_CUDA, "sync");
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_min = std::min(ms_min, ms);
      }
      if (st == VF_OK && ms_min < best) {
        best = ms_min;
        best_ty = tys[ti];
        best_ctas = c;
        best_ppt = b->ppt;
      }
    }
  }
  // the class-kernel form: per class, its class kernel or one launch per
  // image, whichever is faster alone; then the whole form
  int best_mode = VF_BATCH_ONE_KERNEL;
  for (size_t i = 0; i < b->classes.size() && st == VF_OK; ++i) {
    float t[2] = {1e30f, 1e30f};
    for (int form = 0; form < 2 && st == VF_OK; ++form) {
      b->classes[i].per_image = form;
      if (enqueue_one_class(b, i, s) != cudaSuccess) st = set_error(b->ctx, VF_ERR_CUDA, "launch");
      for (int r = 0; r < 3 && st == VF_OK; ++r) {
        cudaEventRecord(e0, s);
        if (enqueue_one_class(b, i, s) != cudaSuccess) st = set_error(b->ctx, VF_ERR_CUDA, "launch");
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = set_error(b->ctx, VF_ERR_CUDA, "sync");
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        t[form] = std::min(t[form], ms);
      }
    }
    b->classes[i].per_image = t[1] < t[0];
  }
  if (st == VF_OK) {
    b->mode = VF_BATCH_CLASS_KERNELS;
    st = enqueue(b, s);  // warm-up
    float ms_min = 1e30f;
    for (int r = 0; r < 3 && st == VF_OK; ++r) {
      cudaEventRecord(e0, s);
      st = enqueue(b, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = set_error(b->ctx, VF_ERR_CUDA, "sync");
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms_min = std::min(ms_min, ms);
    }
    if (st == VF_OK && ms_min < best) {
      best = ms_min;
      best_mode = VF_BATCH_CLASS_KERNELS;
    }
    b->mode = VF_BATCH_ONE_KERNEL;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->ppt = best_ppt;
  if (st != VF_OK) return st;
  st = upload(b, best_ty);
  b->ctas_per_sm = best_ctas;
  b->mode = best_mode;
  drop_graph(b);
  if (tile_rows) *tile_rows = best_ty;
  if (ctas_per_sm) *ctas_per_sm = best_ctas;
  if (best_ms) *best_ms = best;
  return st;
}

vf_status vf_batch_configure(vf_batch* b, int tile_rows, int ctas_per_sm) {
  if (!b) return VF_ERR_ARG;
  if (tile_rows != 2 && tile_rows != 4 && tile_rows != 8)
    return set_error(b->ctx, VF_ERR_ARG, "tile_rows must be 2, 4 or 8");
  if (ctas_per_sm < 0 || ctas_per_sm > resident_ctas(b, tile_rows))
    return set_error(b->ctx, VF_ERR_ARG, "more CTAs per SM than can be resident");
  vf_status st = upload(b, tile_rows);
  b->ctas_per_sm = ctas_per_sm;
  b->mode = VF_BATCH_ONE_KERNEL;  // a configuration of the one-kernel form selects it
  drop_graph(b);
  return st;
}

vf_status vf_batch_set_pixels_per_thread(vf_batch* b, int pixels_per_thread) {
  if (!b) return VF_ERR_ARG;
  if (pixels_per_thread < 0 || pixels_per_thread > 2)
    return set_error(b->ctx, VF_ERR_ARG, "pixels per thread must be 0, 1 or 2");
  b->ppt = pixels_per_thread;
  vf_status st = upload(b, b->ty);
  b->mode = VF_BATCH_ONE_KERNEL;
  drop_graph(b);
  return st;
}

vf_status vf_batch_set_mode(vf_batch* b, int mode) {
  if (!b) return VF_ERR_ARG;
  if (mode != VF_BATCH_ONE_KERNEL && mode != VF_BATCH_CLASS_KERNELS)
    return set_error(b->ctx, VF_ERR_ARG, "mode must be VF_BATCH_ONE_KERNEL or VF_BATCH_CLASS_KERNELS");
  b->mode = mode;
  drop_graph(b);
  return VF_OK;
}

vf_status vf_batch_get_mode(const vf_batch* b, int* mode) {
  if (!b || !mode) return VF_ERR_ARG;
  *mode = b->mode;
  return VF_OK;
}

vf_status vf_batch_get_config(const vf_batch* b, int* tile_rows, int* ctas_per_sm,
                              int* pixels_per_thread) {
  if (!b) return VF_ERR_ARG;
  if (tile_rows) *tile_rows = b->ty;
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  if (pixels_per_thread) *pixels_per_thread = b->ppt;
  return VF_OK;
}

void vf_batch_destroy(vf_batch* b) {
  if (!b) return;
  drop_graph(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->d_imgs) cudaFree(b->d_imgs);
  if (b->d_begin) cudaFree(b->d_begin);
  if (b->d_counter) cudaFree(b->d_counter);
  for (int i = 0; i < kBatchBranches; ++i) {
    if (b->branch[i]) {
      cudaStreamSynchronize(b->branch[i]);
      cudaStreamDestroy(b->branch[i]);
    }
    if (b->join[i]) cudaEventDestroy(b->join[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->d_cimgs) cudaFree(b->d_cimgs);
  if (b->d_cbegin) cudaFree(b->d_cbegin);
  if (b->d_ccounters) cudaFree(b->d_ccounters);
  delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free batched call.  The paper has no counterpart: this serves
// callers that cannot allocate device memory while they filter.  Its scratch
// (the tile counter, the tile prefix array and the image descriptors) lives in
// one file-scope device array of fixed size instead of memory from cudaMalloc;
// everything else is the batch kernel above, in its default configuration
// (32 x 4 tiles, the occupancy maximum of resident CTAs).
#include <mutex>

namespace {

constexpr int kStaticMax = VF_STATIC_MAX_IMAGES;
constexpr int kStaticDevices = 64;

struct StaticLayout {
  unsigned int counter[64];       // [0]: the tile counter (256 bytes keep what follows aligned)
  int begin[kStaticMax + 64];     // first tile of every queued image, then the total
  BatchImage imgs[kStaticMax];    // descriptors in queue order
};

// The scratch itself.  Host code must not pass &g_static_scratch to a kernel:
// on the host the name is a stand-in, not a device address.  The address comes
// from cudaGetSymbolAddress, once per device (static_scratch below).
static __device__ __align__(256) unsigned char g_static_scratch[sizeof(StaticLayout)];

std::mutex g_static_mutex;        // serialises the host side of the calls
StaticLayout g_static_host;       // host staging of begin[] and imgs[]
int g_static_order[kStaticMax];
double g_static_cost[kStaticMax];
void* g_static_dev[kStaticDevices] = {};

// Device address of the scratch on the current device (set up on first use).
vf_status static_scratch(StaticLayout** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VF_ERR_CUDA;
  if (dev < 0 || dev >= kStaticDevices) return VF_ERR_UNSUPPORTED;
  if (!g_static_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return VF_ERR_CUDA;
    }
    g_static_dev[dev] = p;
  }
  *out = static_cast<StaticLayout*>(g_static_dev[dev]);
  return VF_OK;
}

// The checks and the Launch block of vf_filter, without recording error text
// and without fitting: a polynomial must already be in the context's cache.
vf_status static_prepare(const vf_ctx* ctx, const vf_image_desc& d, BatchImage* out,
                         LaunchClass* cls) {
  const vf_params* p = &d.params;
  if (!d.d_in || !d.d_out) return VF_ERR_ARG;
  if (d.height < 1 || d.width < 1 || (d.channels != 3 && d.channels != 4)) return VF_ERR_ARG;
  const size_t row = (size_t)d.width * d.channels;
  if (d.in_pitch < row || d.out_pitch < row) return VF_ERR_ARG;
  if ((int)p->criterion < 0 || (int)p->criterion > 5 || (int)p->approx < 0 || (int)p->approx > 3 ||
      (int)p->precision < 0 || (int)p->precision > 2)
    return VF_ERR_ARG;
  if (p->criterion == VF_EVBDF) return VF_ERR_UNSUPPORTED;
  if (p->window < 1 || (p->window & 1) == 0 || p->window > 15) return VF_ERR_ARG;
  if (p->window != 3 && p->window != 5 && p->window != 7) return VF_ERR_UNSUPPORTED;
  if (p->approx == VF_MINIMAX_POLY && (p->degree < 2 || p->degree > 6)) return VF_ERR_ARG;
  if (p->approx == VF_MINIMAX_RATIONAL_FIT && (p->degree < 2 || p->degree > 4)) return VF_ERR_ARG;
  if (!(p->kappa >= 0.0f) || !(p->exp_cutoff > 0.0f)) return VF_ERR_ARG;
  if (p->precision != VF_FP32) return VF_ERR_UNSUPPORTED;
  const size_t in_bytes = (size_t)(d.height - 1) * d.in_pitch + row;
  const size_t out_bytes = (size_t)(d.height - 1) * d.out_pitch + row;
  if (d.d_in < d.d_out + out_bytes && d.d_out < d.d_in + in_bytes) return VF_ERR_ALIAS;
  const int w = p->window, n = w * w, crit = (int)p->criterion;
  const bool rfit = p->approx == VF_MINIMAX_RATIONAL_FIT;
  int apx = crit == kVMF ? kExact : (rfit ? kRational : (int)p->approx);
  if (apx == kRational && crit == kBVDF) return VF_ERR_UNSUPPORTED;
  Launch& L = out->L;
  L = Launch{};
  L.in = d.d_in;
  L.out = d.d_out;
  L.height = d.height;
  L.width = d.width;
  L.channels = d.channels;
  L.vec4_in = d.channels == 4 && ((uintptr_t)d.d_in % 4 == 0) && d.in_pitch % 4 == 0;
  L.vec4_out = d.channels == 4 && ((uintptr_t)d.d_out % 4 == 0) && d.out_pitch % 4 == 0;
  L.in_pitch = (long long)d.in_pitch;
  L.out_pitch = (long long)d.out_pitch;
  L.kappa_scale = (float)std::pow((double)n, -(double)p->kappa / 3.0);
  L.exp_cutoff = p->exp_cutoff;
  L.ent_cutoff = p->ent_cutoff < 0.0f ? (n <= 9 ? 0.05f : 0.05f * 9.0f / (float)n) : p->ent_cutoff;
  L.stats = nullptr;
  auto put = [](float* dst, const double* src, int len) {
    for (int k = 0; k < 8; ++k) dst[k] = k < len ? (float)src[k] : 0.0f;
  };
  if (apx == kExact && crit == kBVDF) {  // fitted when the context was made
    const double* a = cached_fit(ctx, VF_FN_HALF_ANGLE, kHalfAngleDegree, 0.0, 1.0);
    if (!a) return VF_ERR_UNSUPPORTED;
    put(L.c.a, a, kHalfAngleDegree + 1);
  }
  if (apx == kPoly) {
    const double *a = nullptr, *b = nullptr;
    if (crit == kBVDF) {
      a = cached_fit(ctx, 0, p->degree, 0.0, 0.5);
      b = cached_fit(ctx, 1, p->degree, 0.0, 1.0 / std::sqrt(2.0));
      if (!a || !b) return VF_ERR_UNSUPPORTED;
      put(L.c.b, b, p->degree + 1);
    } else if (crit == kEVMF) {
      if (!(L.ent_cutoff > 0.0f) || L.ent_cutoff >= 1.0f) return VF_ERR_ARG;
      a = cached_fit(ctx, 3, p->degree, (double)L.ent_cutoff, 1.0);
    } else {
      a = cached_fit(ctx, 2, p->degree, 0.0, (double)p->exp_cutoff);
    }
    if (!a) return VF_ERR_UNSUPPORTED;
    put(L.c.a, a, p->degree + 1);
  } else if (apx == kRational && rfit) {
    if (crit == kEVMF && (!(L.ent_cutoff > 0.0f) || L.ent_cutoff >= 1.0f)) return VF_ERR_ARG;
    const double *num = nullptr, *den = nullptr;
    const bool ok = crit == kEVMF
                        ? cached_rational_fit(ctx, 3, p->degree, (double)L.ent_cutoff, 1.0, &num, &den)
                        : cached_rational_fit(ctx, 2, p->degree, 0.0, (double)p->exp_cutoff, &num,
                                              &den);
    if (!ok) return VF_ERR_UNSUPPORTED;
    put(L.c.a, num, p->degree + 1);
    put(L.c.b, den, p->degree + 1);
  } else if (apx == kRational) {
    if ((crit == kAMNFE || crit == kAMNFG) && p->exp_cutoff != 10.0f) return VF_ERR_UNSUPPORTED;
    const double *num = nullptr, *den = nullptr;
    paper_rational(crit == kEVMF ? 3 : 2, &num, &den);
    put(L.c.a, num, 5);
    put(L.c.b, den, 5);
  }
  cls->crit = crit;
  cls->w = w;
  cls->apx = apx;
  cls->deg = p->degree;
  out->cls = class_of(w, crit, apx);
  return VF_OK;
}

}  // namespace

extern "C" {

vf_status vf_batch_run_static(vf_ctx* ctx, const vf_image_desc* descs, int count, void* stream) {
  if (!ctx || !descs || count < 1) return VF_ERR_ARG;
  if (count > kStaticMax) return VF_ERR_UNSUPPORTED;
  // the descriptor copies read the library's one host staging buffer: a
  // captured copy would read it again at every replay, after later calls had
  // overwritten it, so a capturing stream is refused
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &capture) != cudaSuccess) {
    cudaGetLastError();
    return VF_ERR_CUDA;
  }
  if (capture != cudaStreamCaptureStatusNone) return VF_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  StaticLayout* dev = nullptr;
  vf_status st = static_scratch(&dev);
  if (st != VF_OK) return st;
  StaticLayout& H = g_static_host;
  LaunchClass cls[kStaticMax];
  BatchImage* staged = H.imgs;  // filled in descriptor order, then reordered below
  static BatchImage unordered[kStaticMax];
  for (int i = 0; i < count; ++i) {
    st = static_prepare(ctx, descs[i], &unordered[i], &cls[i]);
    if (st != VF_OK) return st;
    g_static_cost[i] = pixel_cost(cls[i]);
    g_static_order[i] = i;
  }
  // queue order: costliest class first, ties by position (std::sort: in place)
  std::sort(g_static_order, g_static_order + count, [](int a, int b) {
    if (g_static_cost[a] != g_static_cost[b]) return g_static_cost[a] > g_static_cost[b];
    return a < b;
  });
  const int ty = 4;
  size_t smem = 0;
  long long total = 0;
  for (int q = 0; q < count; ++q) {
    const int i = g_static_order[q];
    staged[q] = unordered[i];
    Launch& L = staged[q].L;
    staged[q].two = batch_two(0, cls[i].w, cls[i].crit);
    const int rows = ty * (staged[q].two ? 2 : 1);
    L.tiles_x = (L.width + kTX - 1) / kTX;
    H.begin[q] = (int)total;
    total += (long long)L.tiles_x * ((L.height + rows - 1) / rows);
    if (total > 0x7fffffffLL) return VF_ERR_UNSUPPORTED;
    smem = std::max(smem, class_smem(cls[i].w, cls[i].crit, ty, staged[q].two));
  }
  H.begin[count] = (int)total;
  cudaStream_t s = (cudaStream_t)stream;
  int device = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess && smem > 48 * 1024)
    e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kTX * ty, smem);
  // pageable host -> device copies return once the source has been staged, so
  // the host staging may be reused by the next call
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dev->begin, H.begin, sizeof(int) * (count + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dev->imgs, H.imgs, sizeof(BatchImage) * count, cudaMemcpyHostToDevice, s);
  // every call starts its tile counter at zero (the array keeps the last call's)
  if (e == cudaSuccess) e = cudaMemsetAsync(dev->counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) {
    cudaGetLastError();  // leave no error behind for the caller's next CUDA call
    return VF_ERR_CUDA;
  }
  batch_kernel<<<sms * std::max(per_sm, 1), kTX * ty, smem, s>>>(dev->imgs, dev->begin, count,
                                                                 dev->counter);
  return cudaGetLastError() == cudaSuccess ? VF_OK : VF_ERR_CUDA;
}

}  // extern "C"
