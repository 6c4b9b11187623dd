// vf_gate.cu -- the learned impulse detector ("gate"): a 3-layer 3x3
// convolutional network (3 -> 16 -> 16 -> 1 channels, ReLU, sigmoid) that
// flags the pixels worth filtering, its training kernels (forward, backward,
// Adam) and its fused inference kernel.  Not in the paper: it is a learned
// stand-in for the detection step of switching filters (Sec. 3.3's EVMF
// switch decides the same thing with an entropy test).
//
// Arithmetic: BF16 weights (rounded from FP32 master weights after every
// update), FP32 activations and FP32 accumulation.  Convolutions are
// cross-correlations with zero padding, input x0 = RGB / 255 - 1/2.
// Determinism: weight gradients are reduced per CTA into a partial buffer and
// the partials are summed in a fixed order by a second kernel (no floating
// point atomics), so training is bit-reproducible and resumable.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "vf_internal.h"
#include "vf_kernels.cuh"

namespace vf {
cudaError_t launch_gated_w3(const Launch&, const uint8_t*, long long, int, int, int, int, int,
                            cudaStream_t);
cudaError_t launch_gated_w5(const Launch&, const uint8_t*, long long, int, int, int, int, int,
                            cudaStream_t);
cudaError_t launch_gated_w7(const Launch&, const uint8_t*, long long, int, int, int, int, int,
                            cudaStream_t);
cudaError_t launch_sparse_w3(const Launch&, const int*, const unsigned*, unsigned, int, int, int,
                             int, cudaStream_t);
cudaError_t launch_sparse_w5(const Launch&, const int*, const unsigned*, unsigned, int, int, int,
                             int, cudaStream_t);
cudaError_t launch_sparse_w7(const Launch&, const int*, const unsigned*, unsigned, int, int, int,
                             int, cudaStream_t);
}  // namespace vf

namespace {

constexpr int kC = 16;  // hidden channels
constexpr int OFF_W1 = 0, OFF_B1 = 432, OFF_W2 = 448, OFF_B2 = 2752, OFF_W3 = 2768,
              OFF_B3 = 2912, NPARAM = 2913;
static_assert(NPARAM == VF_GATE_NPARAM, "parameter count");
constexpr int kThreads = 256;
constexpr int kWgradBlocks = 64;  // pixel chunks of the weight-gradient reduction

struct Images {
  const uint8_t* img;  // image k at img + k * stride; rows `pitch` bytes apart
  long long stride, pitch;
  int count, H, W, channels;
};

__device__ __forceinline__ float pixel_channel(const Images& I, int b, int y, int x, int c) {
  return (float)I.img[b * I.stride + (long long)y * I.pitch + (long long)x * I.channels + c] *
             (1.0f / 255.0f) -
         0.5f;
}

__device__ __forceinline__ void load_weights(const __nv_bfloat16* wb, float* w, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) w[k] = __bfloat162float(wb[k]);
}

// Activation a[c](b, y, x) of the layer feeding a convolution: x0 from the
// image (layer 1) or relu(z) of the previous layer; 0 outside the image.
template <bool FROM_IMG>
__device__ __forceinline__ float act(const Images& I, const float* z, int cin, int b, int c,
                                     int y, int x) {
  if (y < 0 || y >= I.H || x < 0 || x >= I.W) return 0.0f;
  if constexpr (FROM_IMG) {
    return pixel_channel(I, b, y, x, c);
  } else {
    return fmaxf(z[(((long long)b * cin + c) * I.H + y) * I.W + x], 0.0f);
  }
}

// z_out[b][o][y][x] = bias[o] + sum_c sum_{u,v} W[o][c][u][v] a[c](y+u-1, x+v-1)
template <int CIN, int COUT, bool FROM_IMG>
__global__ void __launch_bounds__(kThreads) conv_fwd(Images I, const __nv_bfloat16* wb,
                                                     int off_w, int off_b, const float* zin,
                                                     float* zout) {
  __shared__ float w[COUT * CIN * 9 + COUT];
  load_weights(wb + off_w, w, COUT * CIN * 9);
  load_weights(wb + off_b, w + COUT * CIN * 9, COUT);
  __syncthreads();
  const long long total = (long long)I.count * I.H * I.W;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int b = (int)(idx / ((long long)I.H * I.W));
  const int rem = (int)(idx - (long long)b * I.H * I.W);
  const int y = rem / I.W, x = rem - y * I.W;
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = w[COUT * CIN * 9 + o];
  for (int c = 0; c < CIN; ++c)
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const float a = act<FROM_IMG>(I, zin, CIN, b, c, y + u - 1, x + v - 1);
#pragma unroll
        for (int o = 0; o < COUT; ++o) acc[o] = fmaf(w[((o * CIN + c) * 3 + u) * 3 + v], a, acc[o]);
      }
#pragma unroll
  for (int o = 0; o < COUT; ++o) zout[(((long long)b * COUT + o) * I.H + y) * I.W + x] = acc[o];
}

// Sigmoid, per-pixel BCE (logit form) and dL/dz3 = (p - t) / N.
__global__ void __launch_bounds__(kThreads) bce_head(Images I, const float* z3,
                                                     const uint8_t* target, float* dz3,
                                                     float* prob, float* loss_part) {
  __shared__ float red[kThreads];
  const long long total = (long long)I.count * I.H * I.W;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (idx < total) {
    const float z = z3[idx];
    const float p = 1.0f / (1.0f + expf(-z));
    if (prob) prob[idx] = p;
    if (target) {
      const float t = target[idx] ? 1.0f : 0.0f;
      l = fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))) - t * z;
      dz3[idx] = (p - t) / (float)total;
    }
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss_part) loss_part[blockIdx.x] = red[0];
}

// Fixed-order sum of n partials into out[0] (one CTA).
__global__ void __launch_bounds__(kThreads) sum_partials(const float* part, int n, float scale,
                                                         float* out) {
  __shared__ float red[kThreads];
  float s = 0.0f;
  for (int k = threadIdx.x; k < n; k += kThreads) s += part[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] * scale;
}

// Weight gradients of one convolution: block (chunk, o * CIN + c) accumulates
// dW[o][c][.][.] (and db[o] when c = 0) over its chunk of pixels into
// part[chunk][...] (a full parameter vector per chunk).
template <int CIN, int COUT, bool FROM_IMG>
__global__ void __launch_bounds__(kThreads) conv_wgrad(Images I, const float* zin,
                                                       const float* dz, int off_w, int off_b,
                                                       float* part) {
  __shared__ float red[10][kThreads];
  const int o = blockIdx.y / CIN, c = blockIdx.y - o * CIN;
  const long long total = (long long)I.count * I.H * I.W;
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  const long long p0 = (long long)blockIdx.x * per, p1 = min(total, p0 + per);
  float g[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) g[k] = 0.0f;
  for (long long idx = p0 + threadIdx.x; idx < p1; idx += kThreads) {
    const int b = (int)(idx / ((long long)I.H * I.W));
    const int rem = (int)(idx - (long long)b * I.H * I.W);
    const int y = rem / I.W, x = rem - y * I.W;
    const float d = dz[(((long long)b * COUT + o) * I.H + y) * I.W + x];
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int v = 0; v < 3; ++v)
        g[u * 3 + v] = fmaf(d, act<FROM_IMG>(I, zin, CIN, b, c, y + u - 1, x + v - 1), g[u * 3 + v]);
    g[9] += d;
  }
#pragma unroll
  for (int k = 0; k < 10; ++k) red[k][threadIdx.x] = g[k];
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
#pragma unroll
      for (int k = 0; k < 10; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 9)
    part[(long long)blockIdx.x * NPARAM + off_w + (o * CIN + c) * 9 + threadIdx.x] =
        red[threadIdx.x][0];
  if (threadIdx.x == 9 && c == 0) part[(long long)blockIdx.x * NPARAM + off_b + o] = red[9][0];
}

// dz_prev[c](q) = [z_prev[c](q) > 0] * sum_o sum_{u,v} W[o][c][u][v] dz[o](q - (u,v) + 1)
template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads) conv_igrad(Images I, const __nv_bfloat16* wb,
                                                       int off_w, const float* dz,
                                                       const float* zprev, float* dzprev) {
  __shared__ float w[COUT * CIN * 9];
  load_weights(wb + off_w, w, COUT * CIN * 9);
  __syncthreads();
  const long long total = (long long)I.count * I.H * I.W;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int b = (int)(idx / ((long long)I.H * I.W));
  const int rem = (int)(idx - (long long)b * I.H * I.W);
  const int y = rem / I.W, x = rem - y * I.W;
  float acc[CIN];
#pragma unroll
  for (int c = 0; c < CIN; ++c) acc[c] = 0.0f;
  for (int o = 0; o < COUT; ++o)
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const int yy = y - u + 1, xx = x - v + 1;
        if (yy < 0 || yy >= I.H || xx < 0 || xx >= I.W) continue;
        const float d = dz[(((long long)b * COUT + o) * I.H + yy) * I.W + xx];
#pragma unroll
        for (int c = 0; c < CIN; ++c) acc[c] = fmaf(w[((o * CIN + c) * 3 + u) * 3 + v], d, acc[c]);
      }
#pragma unroll
  for (int c = 0; c < CIN; ++c) {
    const long long k = (((long long)b * CIN + c) * I.H + y) * I.W + x;
    dzprev[k] = zprev[k] > 0.0f ? acc[c] : 0.0f;
  }
}

// grad[k] = sum over chunks (fixed order), k = 0 .. NPARAM-1
__global__ void reduce_grads(const float* part, int chunks, float* grad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NPARAM) return;
  float s = 0.0f;
  for (int j = 0; j < chunks; ++j) s += part[(long long)j * NPARAM + k];
  grad[k] = s;
}

// Adam (Kingma & Ba, 2015) on the FP32 masters, then the BF16 copy.
__global__ void adam(float* theta, float* m, float* v, const float* grad, __nv_bfloat16* wb,
                     float lr, float b1, float b2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NPARAM) return;
  const float g = grad[k];
  const float mk = b1 * m[k] + (1.0f - b1) * g;
  const float vk = b2 * v[k] + (1.0f - b2) * g * g;
  m[k] = mk;
  v[k] = vk;
  const float t = theta[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  theta[k] = t;
  wb[k] = __float2bfloat16_rn(t);
}

__global__ void to_bf16(const float* theta, __nv_bfloat16* wb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < NPARAM) wb[k] = __float2bfloat16_rn(theta[k]);
}

// ---- fused inference: 32 x 8 outputs per CTA, the three layers in shared
// memory (halo 3 / 2 / 1), activations outside the image are 0 at every layer
constexpr int IX = 32, IY = 8;
constexpr int S0X = IX + 6, S0Y = IY + 6;  // input region
constexpr int S1X = IX + 4, S1Y = IY + 4;  // layer-1 outputs
constexpr int S2X = IX + 2, S2Y = IY + 2;  // layer-2 outputs
constexpr size_t kInferSmem =
    sizeof(float) * (NPARAM + 3 * S0Y * S0X + kC * S1Y * S1X + kC * S2Y * S2X);

__global__ void __launch_bounds__(IX * IY) gate_infer(Images I, const __nv_bfloat16* wb,
                                                      float logit_threshold, uint8_t* flags,
                                                      long long flag_pitch, float* prob,
                                                      int tiles_x) {
  extern __shared__ float sm[];
  float* w = sm;                       // weights, W2 and W3 as [c][u][v][o] for broadcast
  float* s0 = w + NPARAM;              // [3][S0Y][S0X]
  float* s1 = s0 + 3 * S0Y * S0X;      // [16][S1Y][S1X]
  float* s2 = s1 + kC * S1Y * S1X;     // [16][S2Y][S2X]
  const int x0 = (blockIdx.x % tiles_x) * IX, y0 = (blockIdx.x / tiles_x) * IY;
  for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) {
    int dst = k;
    if (k >= OFF_W2 && k < OFF_B2) {  // [o][c][u][v] -> [c][u][v][o]
      int r = k - OFF_W2, o = r / 144, cuv = r - o * 144;
      dst = OFF_W2 + cuv * kC + o;
    }
    w[dst] = __bfloat162float(wb[k]);
  }
  for (int k = threadIdx.x; k < 3 * S0Y * S0X; k += blockDim.x) {
    int c = k / (S0Y * S0X), r = k - c * S0Y * S0X, ry = r / S0X, rx = r - ry * S0X;
    int gy = y0 - 3 + ry, gx = x0 - 3 + rx;
    s0[k] = (gy >= 0 && gy < I.H && gx >= 0 && gx < I.W) ? pixel_channel(I, 0, gy, gx, c) : 0.0f;
  }
  __syncthreads();
  // layer 1 on the S1 region
  for (int k = threadIdx.x; k < S1Y * S1X; k += blockDim.x) {
    int ry = k / S1X, rx = k - ry * S1X;
    int gy = y0 - 2 + ry, gx = x0 - 2 + rx;
    bool in = gy >= 0 && gy < I.H && gx >= 0 && gx < I.W;
    float acc[kC];
#pragma unroll
    for (int o = 0; o < kC; ++o) acc[o] = w[OFF_B1 + o];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          float a = s0[(c * S0Y + ry + u) * S0X + rx + v];
#pragma unroll
          for (int o = 0; o < kC; ++o) acc[o] = fmaf(w[OFF_W1 + ((o * 3 + c) * 3 + u) * 3 + v], a, acc[o]);
        }
#pragma unroll
    for (int o = 0; o < kC; ++o) s1[(o * S1Y + ry) * S1X + rx] = in ? fmaxf(acc[o], 0.0f) : 0.0f;
  }
  __syncthreads();
  // layer 2 on the S2 region
  for (int k = threadIdx.x; k < S2Y * S2X; k += blockDim.x) {
    int ry = k / S2X, rx = k - ry * S2X;
    int gy = y0 - 1 + ry, gx = x0 - 1 + rx;
    bool in = gy >= 0 && gy < I.H && gx >= 0 && gx < I.W;
    float acc[kC];
#pragma unroll
    for (int o = 0; o < kC; ++o) acc[o] = w[OFF_B2 + o];
    for (int c = 0; c < kC; ++c)
#pragma unroll
      for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          float a = s1[(c * S1Y + ry + u) * S1X + rx + v];
          const float* wc = w + OFF_W2 + ((c * 3 + u) * 3 + v) * kC;
#pragma unroll
          for (int o = 0; o < kC; ++o) acc[o] = fmaf(wc[o], a, acc[o]);
        }
#pragma unroll
    for (int o = 0; o < kC; ++o) s2[(o * S2Y + ry) * S2X + rx] = in ? fmaxf(acc[o], 0.0f) : 0.0f;
  }
  __syncthreads();
  // layer 3: one output per thread
  const int tx = threadIdx.x % IX, ty = threadIdx.x / IX;
  const int gx = x0 + tx, gy = y0 + ty;
  float z = w[OFF_B3];
  for (int c = 0; c < kC; ++c)
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int v = 0; v < 3; ++v)
        z = fmaf(w[OFF_W3 + (c * 3 + u) * 3 + v], s2[(c * S2Y + ty + u) * S2X + tx + v], z);
  if (gx < I.W && gy < I.H) {
    if (flags) flags[(long long)gy * flag_pitch + gx] = z > logit_threshold ? 1 : 0;
    if (prob) prob[(long long)gy * I.W + gx] = 1.0f / (1.0f + expf(-z));
  }
}

// ---- fused inference on the tensor cores: each convolution is an implicit
// GEMM (rows = output cells, K = input channel x 3 x 3 taps, N = 16 output
// channels) run with warp-level mma.sync m16n8k16, BF16 operands (activations
// rounded to BF16 between layers), FP32 accumulation.  32 x 16 outputs per
// CTA of 512 threads (halo 3 / 2 / 1 as in gate_infer; the taller tile
// recomputes fewer halo cells per output: 1.41 layer-1 and 1.20 layer-2 cells
// instead of 1.69 and 1.33 at 32 x 8); activations live in shared memory as
// BF16 [cell][channel] so an A fragment is two 32-bit loads per row.
constexpr int TX = 32, TY = 16;                  // outputs per CTA
constexpr int T0X = TX + 6, T0Y = TY + 6;        // input region
constexpr int T1X = TX + 4, T1Y = TY + 4;        // layer-1 cells
constexpr int T2X = TX + 2, T2Y = TY + 2;        // layer-2 cells
constexpr int TC_THREADS = TX * TY;
constexpr int TC_WARPS = TC_THREADS / 32;
constexpr int TC_S1 = T1Y * T1X;                 // 720 layer-1 cells = 45 m-tiles
constexpr int TC_S2 = T2Y * T2X;                 // 612 layer-2 cells
constexpr int TC_S2_TILES = (TC_S2 + 15) / 16;   // 39 m-tiles (the last one partial)
static_assert(TC_S1 % 16 == 0, "whole layer-1 m-tiles");
// dynamic shared memory: BF16 weights (copied once per CTA with 32-bit loads,
// so the B fragments are built from shared memory instead of 2-byte global
// loads), x0, a1, a2, biases; every part 16-byte aligned
constexpr size_t tc_round16(size_t b) { return (b + 15) / 16 * 16; }
constexpr size_t TC_OFF_S0 = tc_round16(NPARAM * 2);
constexpr size_t TC_OFF_S1 = TC_OFF_S0 + tc_round16(3 * T0Y * T0X * 2);
constexpr size_t TC_OFF_S2 = TC_OFF_S1 + (size_t)TC_S1 * kC * 2;
constexpr size_t TC_OFF_BIAS = TC_OFF_S2 + (size_t)TC_S2 * kC * 2;
constexpr size_t TC_SMEM = TC_OFF_BIAS + (2 * kC + 1) * 4;
static_assert(TC_SMEM <= 100 * 1024, "two CTAs per SM");

// Word of channel pair w (0..7) of activation cell `cell`: the two 4-word
// halves of a cell swap places when bit 2 of the cell index is set, so the
// A-fragment loads of 8 consecutive cells x 4 lanes hit 32 distinct banks
// (unswizzled, cells g and g + 4 share banks).
__device__ __forceinline__ int act_word(int cell, int w) {
  return cell * (kC / 2) + (w ^ (cell & 4));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
// max(lo, 0), max(hi, 0) rounded to BF16 and packed (lo in the low half): one
// conversion with ReLU (the rounding keeps the sign, so ReLU before or after
// it gives the same value)
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t bf16_pair(const __nv_bfloat16* w, int i0, int i1) {
  uint32_t lo = *reinterpret_cast<const unsigned short*>(w + i0);
  uint32_t hi = *reinterpret_cast<const unsigned short*>(w + i1);
  return lo | (hi << 16);
}

__global__ void __launch_bounds__(TC_THREADS) gate_infer_tc(Images I, const __nv_bfloat16* wb,
                                                            float logit_threshold, uint8_t* flags,
                                                            long long flag_pitch, float* prob,
                                                            int tiles_x) {
  extern __shared__ __align__(16) unsigned char tc_smem[];
  __nv_bfloat16* sw = reinterpret_cast<__nv_bfloat16*>(tc_smem);            // weights
  __nv_bfloat16* s0 = reinterpret_cast<__nv_bfloat16*>(tc_smem + TC_OFF_S0);  // x0, [c][row][col]
  uint32_t* s1 = reinterpret_cast<uint32_t*>(tc_smem + TC_OFF_S1);  // a1, [cell][16 ch], bf16 pairs
  uint32_t* s2 = reinterpret_cast<uint32_t*>(tc_smem + TC_OFF_S2);  // a2
  float* bias = reinterpret_cast<float*>(tc_smem + TC_OFF_BIAS);
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(wb);  // device_alloc'd: aligned
    uint32_t* dst = reinterpret_cast<uint32_t*>(sw);
    for (int k = threadIdx.x; k < NPARAM / 2; k += blockDim.x) dst[k] = src[k];
    if ((NPARAM & 1) && threadIdx.x == 0) sw[NPARAM - 1] = wb[NPARAM - 1];
  }
  const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  // input region: one pixel per item (a 32-bit load where the layout allows),
  // its three channels scaled as pixel_channel does
  const bool word = I.channels == 4 && (reinterpret_cast<uintptr_t>(I.img) & 3) == 0 &&
                    (I.pitch & 3) == 0;
  for (int k = threadIdx.x; k < T0Y * T0X; k += blockDim.x) {
    const int ry = k / T0X, rx = k - ry * T0X;
    const int gy = y0 - 3 + ry, gx = x0 - 3 + rx;
    float v[3] = {0.0f, 0.0f, 0.0f};
    if (gy >= 0 && gy < I.H && gx >= 0 && gx < I.W) {
      const uint8_t* src = I.img + (long long)gy * I.pitch + (long long)gx * I.channels;
      uint32_t px;
      if (word) px = *reinterpret_cast<const uint32_t*>(src);
      else px = (uint32_t)src[0] | ((uint32_t)src[1] << 8) | ((uint32_t)src[2] << 16);
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c] = (float)((px >> (8 * c)) & 255u) * (1.0f / 255.0f) - 0.5f;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) s0[c * T0Y * T0X + k] = __float2bfloat16_rn(v[c]);
  }
  __syncthreads();  // weights staged
  if (threadIdx.x < kC) bias[threadIdx.x] = __bfloat162float(sw[OFF_B1 + threadIdx.x]);
  else if (threadIdx.x < 2 * kC) bias[threadIdx.x] = __bfloat162float(sw[OFF_B2 + threadIdx.x - kC]);
  else if (threadIdx.x == 2 * kC) bias[threadIdx.x] = __bfloat162float(sw[OFF_B3]);
  __syncthreads();

  // layer 1: K = 27 taps (c, u, v) padded to 32 = two k-steps
  {
    uint32_t b[2][2][2];  // [k-step][n-tile][reg]
    int off[2][4];        // per k-step: s0 offsets of this lane's K columns 2t, 2t+1, 2t+8, 2t+9
    bool kin[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int k = ks * 16 + 2 * t + (e & 1) + (e >> 1) * 8;
        kin[ks][e] = k < 27;
        int c = k / 9, r = k - c * 9, u = r / 3, v = r - u * 3;
        off[ks][e] = kin[ks][e] ? (c * T0Y + u) * T0X + v : 0;
      }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        int n = nt * 8 + g;
        int k0 = ks * 16 + 2 * t, k8 = k0 + 8;
        auto wv = [&](int k) { return k < 27 ? OFF_W1 + n * 27 + k : -1; };
        auto pair = [&](int ka, int kb) {
          uint32_t lo = wv(ka) >= 0 ? *reinterpret_cast<const unsigned short*>(sw + wv(ka)) : 0u;
          uint32_t hi = wv(kb) >= 0 ? *reinterpret_cast<const unsigned short*>(sw + wv(kb)) : 0u;
          return lo | (hi << 16);
        };
        b[ks][nt][0] = pair(k0, k0 + 1);
        b[ks][nt][1] = pair(k8, k8 + 1);
      }
    }
    const unsigned short* s0u = reinterpret_cast<const unsigned short*>(s0);
    for (int mt = warp; mt < TC_S1 / 16; mt += TC_WARPS) {
      float d[2][4] = {};
      const int m0 = mt * 16 + g, m1 = m0 + 8;
      const int base0 = (m0 / T1X) * T0X + m0 % T1X, base1 = (m1 / T1X) * T0X + m1 % T1X;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        uint32_t a[4];
        auto ld = [&](int base, int e) -> uint32_t { return kin[ks][e] ? s0u[base + off[ks][e]] : 0u; };
        a[0] = ld(base0, 0) | (ld(base0, 1) << 16);
        a[1] = ld(base1, 0) | (ld(base1, 1) << 16);
        a[2] = ld(base0, 2) | (ld(base0, 3) << 16);
        a[3] = ld(base1, 2) | (ld(base1, 3) << 16);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) mma_bf16(d[nt], a, b[ks][nt][0], b[ks][nt][1]);
      }
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int m = half ? m1 : m0;
        const int ry = m / T1X, rx = m - ry * T1X;
        const int gy = y0 - 2 + ry, gx = x0 - 2 + rx;
        const bool in = gy >= 0 && gy < I.H && gx >= 0 && gx < I.W;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int n = nt * 8 + 2 * t;
          float v0 = in ? fmaxf(d[nt][half * 2] + bias[n], 0.0f) : 0.0f;
          float v1 = in ? fmaxf(d[nt][half * 2 + 1] + bias[n + 1], 0.0f) : 0.0f;
          s1[act_word(m, n >> 1)] = pack_bf16(v0, v1);
        }
      }
    }
  }
  __syncthreads();

  // layer 2: K = 9 taps x 16 channels = 9 k-steps
  {
    uint32_t b[9][2][2];
#pragma unroll
    for (int ks = 0; ks < 9; ++ks)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int n = nt * 8 + g;  // W2[n][c][u][v], k-step ks = u * 3 + v, c = K column
        const int base = OFF_W2 + n * 144 + ks;
        b[ks][nt][0] = bf16_pair(sw, base + (2 * t) * 9, base + (2 * t + 1) * 9);
        b[ks][nt][1] = bf16_pair(sw, base + (2 * t + 8) * 9, base + (2 * t + 9) * 9);
      }
    for (int mt = warp; mt < TC_S2_TILES; mt += TC_WARPS) {
      float d[2][4] = {};
      const int m0 = mt * 16 + g, m1 = m0 + 8;
      const int c0 = min(m0, TC_S2 - 1), c1 = min(m1, TC_S2 - 1);
      const int base0 = (c0 / T2X) * T1X + c0 % T2X, base1 = (c1 / T2X) * T1X + c1 % T2X;
#pragma unroll
      for (int ks = 0; ks < 9; ++ks) {
        const int o = (ks / 3) * T1X + ks % 3;
        const int ca = base0 + o, cb = base1 + o;
        uint32_t a[4] = {s1[act_word(ca, t)], s1[act_word(cb, t)], s1[act_word(ca, t + 4)],
                         s1[act_word(cb, t + 4)]};
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) mma_bf16(d[nt], a, b[ks][nt][0], b[ks][nt][1]);
      }
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int m = half ? m1 : m0;
        if (m >= TC_S2) continue;
        const int ry = m / T2X, rx = m - ry * T2X;
        const int gy = y0 - 1 + ry, gx = x0 - 1 + rx;
        const bool in = gy >= 0 && gy < I.H && gx >= 0 && gx < I.W;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int n = nt * 8 + 2 * t;
          float v0 = in ? fmaxf(d[nt][half * 2] + bias[kC + n], 0.0f) : 0.0f;
          float v1 = in ? fmaxf(d[nt][half * 2 + 1] + bias[kC + n + 1], 0.0f) : 0.0f;
          s2[act_word(m, n >> 1)] = pack_bf16(v0, v1);
        }
      }
    }
  }
  __syncthreads();

  // layer 3: one output channel (N padded to 8 with zero weights)
  {
    uint32_t b[9][2];
#pragma unroll
    for (int ks = 0; ks < 9; ++ks) {
      const int base = OFF_W3 + ks;  // W3[0][c][u][v]
      b[ks][0] = g == 0 ? bf16_pair(sw, base + (2 * t) * 9, base + (2 * t + 1) * 9) : 0u;
      b[ks][1] = g == 0 ? bf16_pair(sw, base + (2 * t + 8) * 9, base + (2 * t + 9) * 9) : 0u;
    }
    for (int mt = warp; mt < TC_THREADS / 16; mt += TC_WARPS) {
      float d[4] = {};
      const int m0 = mt * 16 + g, m1 = m0 + 8;  // output pixel (m / TX, m % TX)
      const int base0 = (m0 / TX) * T2X + m0 % TX, base1 = (m1 / TX) * T2X + m1 % TX;
#pragma unroll
      for (int ks = 0; ks < 9; ++ks) {
        const int o = (ks / 3) * T2X + ks % 3;
        const int ca = base0 + o, cb = base1 + o;
        uint32_t a[4] = {s2[act_word(ca, t)], s2[act_word(cb, t)], s2[act_word(ca, t + 4)],
                         s2[act_word(cb, t + 4)]};
        mma_bf16(d, a, b[ks][0], b[ks][1]);
      }
      if (t == 0) {  // column n = 0 of D: d[0] (row g) and d[2] (row g + 8)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int m = half ? m1 : m0;
          const int gx = x0 + m % TX, gy = y0 + m / TX;
          const float z = d[half * 2] + bias[2 * kC];
          if (gx < I.W && gy < I.H) {
            if (flags) flags[(long long)gy * flag_pitch + gx] = z > logit_threshold ? 1 : 0;
            if (prob) prob[(long long)gy * I.W + gx] = 1.0f / (1.0f + expf(-z));
          }
        }
      }
    }
  }
}

// ---- fused inference on the 5th-generation tensor cores (tcgen05): every
// layer is an implicit GEMM over rows of 128 cells (M = 128 cells, K = 16
// input channels), BF16 operands staged in shared memory in the K-major,
// unswizzled core-matrix layout, FP32 accumulators in tensor memory (TMEM):
//   x0  [row][130 cells][8 channels: R, G, B, 0 ...]          (16 B per cell)
//   a1, a2  two such planes per layer (channels 0-7, 8-15)
// A tap's shifted cells are the same planar activations read from a start
// address 16 bytes per cell further on, so no operand is ever gathered.
//
// The three tap rows of a 3 x 3 layer go to the MMA's N dimension instead of
// to separate MMAs.  TMEM columns are blocks of 16, block b the accumulator
// of output row b - 2.  One MMA takes one input row r (one tap column: A
// shifted by 0, 1 or 2 cells) against the weights of all three tap rows laid
// side by side along N in reverse order, and writes blocks r .. r + 2: block
// r + g receives tap row 2 - g, which is exactly input row r's share of
// output row r - 2 + g.  Every MMA accumulates onto its blocks, so the sum
// over tap rows builds up in TMEM as the input rows stream past (a sliding
// accumulator; the blocks are cleared beforehand with tcgen05.st):
//   layer 1 (3 -> 16): K = 8 channels of row r and 8 of row r + 1 (the next
//            K half one row further on), N = 64 (output rows r - 2 .. r + 1):
//            6 row pairs x 3 tap columns = 18 MMAs per tile;
//   layer 2 (16 -> 16): N = 48, 10 rows x 3 tap columns = 30 MMAs;
//   layer 3 (16 -> 1): N = 48 with the tap columns in the first three
//            columns of each block (the others zero weights), the cell
//            shift applied afterwards (the output of cell x adds column v of
//            cell x + v: warp shuffles, and shared memory across the lane
//            quarters): 8 MMAs.
// 56 MMAs per tile instead of 162 with one MMA of N = 16 per tap: at these
// widths an MMA costs the tensor core nearly the same time whatever its N
// (measured: 61 cycles back to back from one thread for N = 16 .. 64, 66 at
// 128), so the count is what bounds the kernel.  A ninth warp only issues
// the MMAs (in order: they accumulate onto shared blocks), each layer in two
// halves committed to mbarriers of their own; after the (bounded) wait for a
// half the eight other warps read its finished output rows back with
// tcgen05.ld (warp w: TMEM lanes 32 (w mod 4) .. + 31, the blocks of one
// parity), add the bias, apply ReLU, round to BF16 and write the next
// layer's planes, then clear the blocks they own -- while the second half's
// MMAs run.  Outputs per CTA tile:
// 124 x 6 (the 128-cell rows shrink by two cells per layer); two CTAs per
// SM, persistent over the tiles.  Numerics as gate_infer_tc: BF16 input and
// activations between layers, BF16 weights, FP32 accumulation and biases.
constexpr int G5_X = 124, G5_Y = 6;                    // outputs per tile (8: no faster)
constexpr int G5_CW = 130;                             // cells per staged row
constexpr int G5_RP = G5_CW * 16;                      // bytes per staged row
constexpr int G5_R0 = G5_Y + 6, G5_R1 = G5_Y + 4, G5_R2 = G5_Y + 2;  // rows of x0, a1, a2
// the halves of each layer: layer 1's first half takes the x0 row pairs below
// G5_H1 and completes output rows [0, G5_O1); layer 2's first half takes a1
// rows [0, G5_O1) and completes rows [0, G5_O2); layer 3's a2 rows [0, G5_O2)
constexpr int G5_H1 = 2 * ((G5_R0 / 2 + 1) / 2), G5_O1 = G5_H1 - 2, G5_O2 = G5_O1 - 2;
static_assert(G5_Y % 2 == 0 && G5_O2 > 0, "even tile heights, non-empty halves");
constexpr int G5_A1P = G5_R1 * G5_RP, G5_A2P = G5_R2 * G5_RP;      // plane bytes
constexpr int G5_N1 = 64, G5_N2 = 48, G5_N3 = 48;      // MMA widths of the layers
constexpr int G5_B1 = 2 * G5_N1 * 16, G5_B2 = 2 * G5_N2 * 16;  // bytes of one B operand
constexpr int G5_OFF_B1 = 0;                           // 3 tap columns each
constexpr int G5_OFF_B2 = G5_OFF_B1 + 3 * G5_B1;
constexpr int G5_OFF_B3 = G5_OFF_B2 + 3 * G5_B2;
constexpr int G5_OFF_BIAS = G5_OFF_B3 + 2 * G5_N3 * 16;
constexpr int G5_OFF_X0 = G5_OFF_BIAS + 256;           // x0, later a2 (x0 is dead by then)
constexpr int G5_OFF_A1 = G5_OFF_X0 + 2 * G5_A2P;
constexpr int G5_RAW_CW = G5_CW + 2;                  // raw cells per row: xs - 4 .. xs + 127
constexpr int G5_OFF_RAW = G5_OFF_A1 + 2 * G5_A1P;      // the next tile's pixels (32-bit)
constexpr int G5_SMEM = G5_OFF_RAW + G5_R0 * G5_RAW_CW * 4;
static_assert(G5_X % 4 == 0 && G5_RAW_CW % 4 == 0, "raw rows are whole 16-byte chunks");
constexpr int G5_THREADS = 256;                        // epilogue threads (eight warps)
constexpr int G5_BLOCK = G5_THREADS + 32;              // and one warp that issues the MMAs
constexpr int G5_BLOCKS = G5_R0 + 2;                   // TMEM blocks (output rows -2 .. R0 - 1)
constexpr int G5_TMEM_COLS = 256;
static_assert(G5_R0 * G5_RP <= 2 * G5_A2P, "x0 fits in the a2 planes it shares");
static_assert(G5_SMEM <= 113 * 1024, "two CTAs per SM");
static_assert(16 * G5_BLOCKS <= G5_TMEM_COLS, "the accumulator blocks fit the TMEM allocation");
static_assert(G5_R0 % 2 == 0, "layer 1 takes the x0 rows in pairs");
// instruction descriptor (kind::f16): FP32 D, BF16 A and B, both K-major,
// N / 8 at bits 17-22, M / 16 = 8 (M = 128) at bits 24-28
__host__ __device__ constexpr uint32_t g5_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | (8u << 24);
}

__device__ __forceinline__ uint32_t g5_smem(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// Shared-memory matrix descriptor: start address, leading (K-direction)
// byte offset, stride (M/N-direction, next 8 rows) byte offset, descriptor
// version 1, no swizzle.
__device__ __forceinline__ uint64_t g5_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// D[tmem] += A * B^T (every MMA accumulates: the blocks are cleared first)
template <int N>
__device__ __forceinline__ void g5_mma(uint32_t d_tmem, uint64_t a, uint64_t b) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(g5_idesc(N)), "r"(1));
}
// Bounded wait for the mbarrier phase `parity` (about a second at most);
// false if it gave up.
__device__ __forceinline__ bool g5_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < (1ll << 24); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity));
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void g5_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ uint32_t g5_ld1(uint32_t taddr) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n" : "=r"(r) : "r"(taddr));
  return r;
}
__device__ __forceinline__ void g5_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}
// Clears this warp's accumulator blocks (its 32 lanes, blocks b = h, h + 2,
// ...) and waits for the stores.
__device__ __forceinline__ void g5_clear(uint32_t lane_addr, int h) {
  const uint32_t z = 0u;
  for (int b = h; b < G5_BLOCKS; b += 2)
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
        "%1,%1,%1};\n" ::"r"(lane_addr + 16 * b),
        "r"(z));
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void g5_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void g5_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void g5_proxy_fence() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__global__ void __launch_bounds__(G5_BLOCK, 2)
    gate_infer_tc5(Images I, const __nv_bfloat16* wb, float logit_threshold, uint8_t* flags,
                   long long flag_pitch, float* prob, int tiles_x, int ntiles, int* status) {
  extern __shared__ __align__(128) unsigned char g5[];
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) unsigned long long s_bar[6];  // the two halves of each layer
  __shared__ int s_fail;
  __shared__ float s_edge[G5_Y][4][3];  // layer 3: lanes 0, 1 of each quarter, for lanes 30, 31
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool worker = warp < G5_THREADS / 32;  // the last warp only issues MMAs
  const int q = warp & 3, h = warp >> 2;  // TMEM lane quarter, block parity
  const int cell = 32 * q + lane;         // the cell (TMEM lane) this thread reads back
  float* bias = reinterpret_cast<float*>(g5 + G5_OFF_BIAS);

  // B operands ([K half][n][8 k], 16 bytes per n) and biases, once.  Column
  // group g of an operand (n = 16 g + o) holds tap row 2 - g (layer 1's
  // second K half, the next input row: tap row 3 - g).
  for (int e = tid; worker && e < 3 * G5_N1 * 16 + 3 * G5_N2 * 16 + G5_N3 * 16;
       e += G5_THREADS) {
    int off, nn, idx;
    float v = 0.0f;
    if (e < 3 * G5_N1 * 16) {  // layer 1, tap column tv: K = (row half, channel)
      const int tv = e / (G5_N1 * 16);
      idx = e % (G5_N1 * 16);
      nn = G5_N1;
      off = G5_OFF_B1 + tv * G5_B1;
      const int n = idx >> 4, k = idx & 15, g = n >> 4, o = n & 15, c = k & 7;
      const int u = 2 - g + (k >> 3);
      if (u >= 0 && u <= 2 && c < 3)
        v = __bfloat162float(wb[OFF_W1 + ((o * 3 + c) * 3 + u) * 3 + tv]);
    } else if (e < 3 * G5_N1 * 16 + 3 * G5_N2 * 16) {  // layer 2: K = input channel
      const int e2 = e - 3 * G5_N1 * 16, tv = e2 / (G5_N2 * 16);
      idx = e2 % (G5_N2 * 16);
      nn = G5_N2;
      off = G5_OFF_B2 + tv * G5_B2;
      const int n = idx >> 4, k = idx & 15, g = n >> 4, o = n & 15;
      v = __bfloat162float(wb[OFF_W2 + (o * kC + k) * 9 + (2 - g) * 3 + tv]);
    } else {  // layer 3: column 16 g + tv of block g is tap (2 - g, tv)
      idx = e - 3 * G5_N1 * 16 - 3 * G5_N2 * 16;
      nn = G5_N3;
      off = G5_OFF_B3;
      const int n = idx >> 4, k = idx & 15, g = n >> 4, tv = n & 15;
      if (tv < 3) v = __bfloat162float(wb[OFF_W3 + k * 9 + (2 - g) * 3 + tv]);
    }
    const int n = idx >> 4, k = idx & 15;
    *reinterpret_cast<__nv_bfloat16*>(g5 + off + (k >> 3) * (nn * 16) + n * 16 + (k & 7) * 2) =
        __float2bfloat16_rn(v);
  }
  if (tid < kC) bias[tid] = __bfloat162float(wb[OFF_B1 + tid]);
  else if (tid < 2 * kC) bias[tid] = __bfloat162float(wb[OFF_B2 + tid - kC]);
  else if (tid == 2 * kC) bias[tid] = __bfloat162float(wb[OFF_B3]);
  // the two padding cells of every a1 row (read only by discarded cells)
  for (int e = tid; worker && e < 2 * G5_R1 * 2; e += G5_THREADS) {
    const int plane = e / (2 * G5_R1), r = (e / 2) % G5_R1, c = 128 + (e & 1);
    *reinterpret_cast<uint4*>(g5 + G5_OFF_A1 + plane * G5_A1P + r * G5_RP + c * 16) =
        make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    for (int k = 0; k < 6; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(g5_smem(&s_bar[k])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     g5_smem(&s_taddr)),
                 "r"(G5_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    g5_fence_before();
  }
  __syncthreads();
  g5_fence_after();
  const uint32_t tmem = s_taddr;
  const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
  if (worker) g5_clear(lane_addr, h);  // the first tile's accumulators
  g5_fence_before();
  uint32_t parity = 0;
  const bool word = I.channels == 4 && (reinterpret_cast<uintptr_t>(I.img) & 3) == 0 &&
                    (I.pitch & 3) == 0;
  // descriptors of the operand bases; a start address further on by d bytes
  // (a multiple of 16) is the same descriptor plus d / 16 (the 14-bit address
  // field cannot carry: every address is below 256 KB)
  const uint64_t dx0 = g5_desc(g5_smem(g5 + G5_OFF_X0), G5_RP, 128);
  const uint64_t da1 = g5_desc(g5_smem(g5 + G5_OFF_A1), G5_A1P, 128);
  const uint64_t da2 = g5_desc(g5_smem(g5 + G5_OFF_X0), G5_A2P, 128);
  const uint64_t db1 = g5_desc(g5_smem(g5 + G5_OFF_B1), G5_N1 * 16, 128);
  const uint64_t db2 = g5_desc(g5_smem(g5 + G5_OFF_B2), G5_N2 * 16, 128);
  const uint64_t db3 = g5_desc(g5_smem(g5 + G5_OFF_B3), G5_N3 * 16, 128);
  constexpr uint64_t kCellD = 1, kRowD = G5_RP / 16, kB1D = G5_B1 / 16, kB2D = G5_B2 / 16;
  // the next tile's input pixels, fetched while the tile's last layer runs,
  // into the raw buffer (rows of cells xs - 4 .. xs + 127): RGBX rows in
  // 16-byte chunks by cp.async (zero-filled past the image's right edge)
  // where the image and its pitch are 16-byte aligned, else 32-bit words by
  // cp.async, or 3-byte pixels into registers.  Which cells lie inside the
  // image is decided again from their coordinates when they are staged.
  constexpr int kPre = (G5_R0 * G5_CW + G5_THREADS - 1) / G5_THREADS;
  constexpr int kChunks = G5_R0 * (G5_RAW_CW / 4);
  const bool vec = I.channels == 4 && (reinterpret_cast<uintptr_t>(I.img) & 15) == 0 &&
                   (I.pitch & 15) == 0;
  uint32_t pre[kPre];
  uint32_t* raw = reinterpret_cast<uint32_t*>(g5 + G5_OFF_RAW);
  auto fetch = [&](int t) {
    if (!worker) return;
    const int xs = (t % tiles_x) * G5_X, ys = (t / tiles_x) * G5_Y;
    if (vec) {
      for (int j = tid; j < kChunks; j += G5_THREADS) {
        const int r = j / (G5_RAW_CW / 4), q = j - r * (G5_RAW_CW / 4);
        const int gy = ys - 3 + r, x = xs - 4 + 4 * q;  // x: a multiple of 4
        int bytes = 0;
        if (t < ntiles && gy >= 0 && gy < I.H && x >= 0) bytes = min(16, max(0, (I.W - x) * 4));
        const uint8_t* src = bytes ? I.img + (long long)gy * I.pitch + 4LL * x : I.img;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(
                         g5_smem(raw + r * G5_RAW_CW + 4 * q)),
                     "l"(src), "r"(bytes)
                     : "memory");
      }
    } else {
#pragma unroll
      for (int j = 0; j < kPre; ++j) {
        const int e = tid + j * G5_THREADS;
        const int r = e / G5_CW, c = e - r * G5_CW;
        const int gy = ys - 3 + r, gx = xs - 3 + c;
        if (e >= G5_R0 * G5_CW || t >= ntiles || gy < 0 || gy >= I.H || gx < 0 || gx >= I.W)
          continue;
        const uint8_t* src = I.img + (long long)gy * I.pitch + (long long)gx * I.channels;
        if (word)
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(
                           g5_smem(raw + r * G5_RAW_CW + c + 1)),
                       "l"(src)
                       : "memory");
        else
          pre[j] = (uint32_t)src[0] | ((uint32_t)src[1] << 8) | ((uint32_t)src[2] << 16);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  // Each layer's MMAs go out in two halves, each committed to its own
  // mbarrier: the epilogue of the first half's finished output rows runs
  // while the second half's MMAs do (and the next layer's first half while
  // the epilogue of the second).  Thread 0 issues (in order: the halves
  // accumulate onto shared blocks) right after a barrier that published the
  // operands; every thread then waits on the mbarrier itself (bounded; a
  // wait that gives up marks the tile failed and the loop stops).
  auto publish = [&] {  // operands (generic proxy) and cleared blocks, for the MMAs
    g5_fence_before();
    g5_proxy_fence();
    __syncthreads();
  };
  auto issue = [&](int k, auto mmas) {
    if (tid == G5_THREADS) {
      g5_fence_after();
      mmas();
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              g5_smem(&s_bar[k])));
    }
  };
  auto await = [&](int k) {
    if (!worker) return;
    if (!g5_wait(g5_smem(&s_bar[k]), parity)) s_fail = 1;
    g5_fence_after();
  };
  // clears this warp's blocks (parity h) among [lo, hi)
  auto clear = [&](int lo, int hi) {
    if (!worker) return;
    const uint32_t z = 0u;
    for (int b = lo + ((h - lo) & 1); b < hi; b += 2)
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
          "%1,%1,%1,%1};\n" ::"r"(lane_addr + 16 * b),
          "r"(z));
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
  };

  bool ok = true;
  fetch(blockIdx.x);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();  // the first tile's raw pixels, copied by every thread
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int xs = (tile % tiles_x) * G5_X, ys = (tile / tiles_x) * G5_Y;
    // x0 rows ys - 3 .. ys + G5_Y + 2, cells xs - 3 .. xs + 126 (zero outside
    // the image), from the pixels fetched during the previous tile
#pragma unroll
    for (int j = 0; j < kPre; ++j) {
      const int e = tid + j * G5_THREADS;
      if (!worker || e >= G5_R0 * G5_CW) break;
      const int r = e / G5_CW, c = e - r * G5_CW;
      const int gy = ys - 3 + r, gx = xs - 3 + c;
      const uint32_t px = (vec || word) ? raw[r * G5_RAW_CW + c + 1] : pre[j];
      uint32_t w01 = 0u, w23 = 0u;
      if (gy >= 0 && gy < I.H && gx >= 0 && gx < I.W) {
        // byte k as the FP32 number 2^23 + byte (one byte permute) minus 2^23:
        // the byte's value exactly, without an integer-to-float conversion
        auto chan = [&](uint32_t sel) {
          return __uint_as_float(__byte_perm(px, 0x4B000000u, sel)) - 8388608.0f;
        };
        const float cr = chan(0x7540u) * (1.0f / 255.0f) - 0.5f;
        const float cg = chan(0x7541u) * (1.0f / 255.0f) - 0.5f;
        const float cb = chan(0x7542u) * (1.0f / 255.0f) - 0.5f;
        w01 = pack_bf16(cr, cg);
        w23 = pack_bf16(cb, 0.0f);
      }
      *reinterpret_cast<uint4*>(g5 + G5_OFF_X0 + r * G5_RP + c * 16) = make_uint4(w01, w23, 0u, 0u);
    }
    // layer 1: x0 row pairs (r, r + 1), r even, into blocks r .. r + 3; the
    // first half (x0 rows 0-5) completes output rows 0-3 (blocks 2-5)
    publish();
    issue(0, [&] {
      for (int r = 0; r < G5_H1; r += 2)
        for (int v = 0; v < 3; ++v)
          g5_mma<G5_N1>(tmem + 16 * r, dx0 + r * kRowD + v * kCellD, db1 + v * kB1D);
    });
    issue(1, [&] {
      for (int r = G5_H1; r < G5_R0; r += 2)
        for (int v = 0; v < 3; ++v)
          g5_mma<G5_N1>(tmem + 16 * r, dx0 + r * kRowD + v * kCellD, db1 + v * kB1D);
    });
    // output rows [y0, y1) of this thread's parity h, two tcgen05.ld per
    // wait: z + bias, ReLU, BF16, into the next layer's two planes (0
    // outside the image)
    auto act_rows = [&](int y0, int y1, int gy0, int gx0, const float* bs,
                        unsigned char* planes, int plane_bytes) {
      if (!worker) return;
      float b[16];  // in registers: the stores below may not alias them
#pragma unroll
      for (int k = 0; k < 16; ++k) b[k] = bs[k];
      for (int y = y0 + ((h - y0) & 1); y < y1; y += 4) {
        uint32_t z[2][16];
        const bool two = y + 2 < y1;
        g5_ld16(lane_addr + 16 * (y + 2), z[0]);
        if (two) g5_ld16(lane_addr + 16 * (y + 4), z[1]);
        g5_wait_ld();
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          if (i == 1 && !two) break;
          const int yy = y + 2 * i, gy = gy0 + yy, gx = gx0 + cell;
          const bool in = gy >= 0 && gy < I.H && gx >= 0 && gx < I.W;
          uint32_t w[8];
#pragma unroll
          for (int k = 0; k < 8; ++k)
            w[k] = in ? pack_bf16_relu(__uint_as_float(z[i][2 * k]) + b[2 * k],
                                       __uint_as_float(z[i][2 * k + 1]) + b[2 * k + 1])
                      : 0u;
          unsigned char* dst = planes + yy * G5_RP + cell * 16;
          *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
          *reinterpret_cast<uint4*>(dst + plane_bytes) = make_uint4(w[4], w[5], w[6], w[7]);
        }
      }
    };
    // layer 1, first half: a1 rows 0-3; blocks 0-5 cleared (the second
    // half's MMAs write blocks 6-13)
    await(0);
    act_rows(0, G5_O1, ys - 2, xs - 2, bias, g5 + G5_OFF_A1, G5_A1P);
    clear(0, G5_O1 + 2);
    publish();
    // layer 2, first half: a1 rows 0-3 into blocks 0-5 (output rows 0-1 complete)
    issue(2, [&] {
      for (int r = 0; r < G5_O1; ++r)
        for (int v = 0; v < 3; ++v)
          g5_mma<G5_N2>(tmem + 16 * r, da1 + r * kRowD + v * kCellD, db2 + v * kB2D);
    });
    // layer 1, second half: a1 rows 4-9; blocks 6-13 cleared
    await(1);
    act_rows(G5_O1, G5_R1, ys - 2, xs - 2, bias, g5 + G5_OFF_A1, G5_A1P);
    clear(G5_O1 + 2, G5_BLOCKS);
    publish();
    // layer 2, second half: a1 rows 4-9 into blocks 4-11
    issue(3, [&] {
      for (int r = G5_O1; r < G5_R1; ++r)
        for (int v = 0; v < 3; ++v)
          g5_mma<G5_N2>(tmem + 16 * r, da1 + r * kRowD + v * kCellD, db2 + v * kB2D);
    });
    // layer 2, first half: a2 rows 0-1 (over x0, whose MMAs are done);
    // blocks 0-3 cleared
    await(2);
    act_rows(0, G5_O2, ys - 1, xs - 1, bias + kC, g5 + G5_OFF_X0, G5_A2P);
    clear(0, G5_O2 + 2);
    publish();
    // layer 3 (one output channel), first half: a2 rows 0-1, unshifted, into
    // blocks 0-3; column v of output row y's block is the sum over the tap
    // row and channels for tap column v at this cell
    issue(4, [&] {
      for (int r = 0; r < G5_O2; ++r) g5_mma<G5_N3>(tmem + 16 * r, da2 + r * kRowD, db3);
    });
    // layer 2, second half: a2 rows 2-7; blocks 4-13 cleared
    await(3);
    act_rows(G5_O2, G5_R2, ys - 1, xs - 1, bias + kC, g5 + G5_OFF_X0, G5_A2P);
    clear(G5_O2 + 2, G5_BLOCKS);
    publish();
    // layer 3, second half: a2 rows 2-7 into blocks 2-9; the next tile's
    // pixels are fetched while the MMAs run
    issue(5, [&] {
      for (int r = G5_O2; r < G5_R2; ++r) g5_mma<G5_N3>(tmem + 16 * r, da2 + r * kRowD, db3);
    });
    fetch(tile + gridDim.x);
    await(5);
    // logit of cell x: column 0 of cell x + column 1 of cell x + 1 + column 2
    // of cell x + 2 (shuffles; the next lane quarter's first lanes through
    // shared memory)
    const float b3 = bias[2 * kC];
    constexpr int kOut = G5_Y / 2;  // output rows per thread
    float c0[kOut] = {}, c1[kOut] = {}, c2[kOut] = {};
    if (worker) {
#pragma unroll
      for (int i = 0; i < kOut; ++i) {
        const int y = h + 2 * i;
        const uint32_t a = lane_addr + 16 * (y + 2);
        c0[i] = __uint_as_float(g5_ld1(a));
        c1[i] = __uint_as_float(g5_ld1(a + 1));
        c2[i] = __uint_as_float(g5_ld1(a + 2));
      }
      g5_wait_ld();
#pragma unroll
      for (int i = 0; i < kOut; ++i) {
        const int y = h + 2 * i;
        if (lane == 0) {
          s_edge[y][q][0] = c1[i];
          s_edge[y][q][1] = c2[i];
        } else if (lane == 1) {
          s_edge[y][q][2] = c2[i];
        }
      }
    }
    clear(0, G5_R2 + 2);  // the next tile's layer-1 accumulators (the rest are clear)
    g5_fence_before();
    asm volatile("cp.async.wait_all;\n" ::: "memory");  // published by the barrier
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kOut && worker; ++i) {
      const int y = h + 2 * i;
      float s1 = __shfl_down_sync(0xffffffffu, c1[i], 1);
      float s2 = __shfl_down_sync(0xffffffffu, c2[i], 2);
      if (q < 3) {
        if (lane == 31) s1 = s_edge[y][q + 1][0];
        if (lane == 30) s2 = s_edge[y][q + 1][1];
        if (lane == 31) s2 = s_edge[y][q + 1][2];
      }
      const float z = (c0[i] + s1) + s2 + b3;
      const int gy = ys + y, gx = xs + cell;
      if (cell < G5_X && gy < I.H && gx < I.W) {
        if (flags) flags[(long long)gy * flag_pitch + gx] = z > logit_threshold ? 1 : 0;
        if (prob) prob[(long long)gy * I.W + gx] = 1.0f / (1.0f + expf(-z));
      }
    }
    parity ^= 1u;
    __syncthreads();  // the tile's reads of the x0 / a2 planes and of s_edge are done
    ok = s_fail == 0;  // uniform: read after the barrier
  }
  if (!ok) {
    if (tid == 0) atomicExch(status, 1);
    // a wait gave up: before the accumulators are freed, wait once more
    // (bounded) on the tile's last commit, which tracks every MMA issued
    // before it (the tile's phase is parity ^ 1 after the flip above)
    if (worker) g5_wait(g5_smem(&s_bar[5]), parity ^ 1u);
  }
  g5_fence_before();
  __syncthreads();
  if (warp == 0) {
    g5_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(G5_TMEM_COLS));
  }
}

uint32_t crc32(const unsigned char* p, size_t n, uint32_t crc = 0) {
  // CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320), bitwise
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) {
    crc ^= p[i];
    for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
  }
  return ~crc;
}

}  // namespace

using namespace vf;

struct vf_gate {
  vf_ctx* ctx = nullptr;
  float* theta = nullptr;  // FP32 masters
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  __nv_bfloat16* wb = nullptr;
  unsigned long long step = 0, seed = 0;
  // training scratch, grown on demand
  float* z1 = nullptr;
  float* z2 = nullptr;
  float* z3 = nullptr;
  float* dz1 = nullptr;
  float* dz2 = nullptr;
  float* part = nullptr;
  float* loss_part = nullptr;
  long long cap_pixels = 0;
  int* d_status = nullptr;  // 1 after a bounded device-side wait gave up
  int sms = 0;
};

namespace {

void free_scratch(vf_gate* g) {
  for (float** p : {&g->z1, &g->z2, &g->z3, &g->dz1, &g->dz2, &g->loss_part}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  g->cap_pixels = 0;
}

vf_status ensure_scratch(vf_gate* g, long long pixels) {
  if (pixels <= g->cap_pixels) return VF_OK;
  free_scratch(g);
  const size_t P = (size_t)pixels;
  const long long blocks = (pixels + kThreads - 1) / kThreads;
  cudaError_t e = device_alloc(&g->z1, P * kC * 4);
  if (e == cudaSuccess) e = device_alloc(&g->z2, P * kC * 4);
  if (e == cudaSuccess) e = device_alloc(&g->z3, P * 4);
  if (e == cudaSuccess) e = device_alloc(&g->dz1, P * kC * 4);
  if (e == cudaSuccess) e = device_alloc(&g->dz2, P * kC * 4);
  if (e == cudaSuccess) e = device_alloc(&g->loss_part, (size_t)blocks * 4);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_scratch(g);
    return set_error(g->ctx, VF_ERR_OOM, "gate training scratch allocation failed");
  }
  g->cap_pixels = pixels;
  return VF_OK;
}

vf_status check_images(vf_gate* g, const uint8_t* d_imgs, int count, int H, int W, int channels,
                       size_t pitch, Images* I) {
  if (!d_imgs || count < 1 || H < 1 || W < 1 || (channels != 3 && channels != 4) ||
      pitch < (size_t)W * channels)
    return set_error(g->ctx, VF_ERR_ARG, "bad gate images");
  I->img = d_imgs;
  I->pitch = (long long)pitch;
  I->stride = (long long)pitch * H;
  I->count = count;
  I->H = H;
  I->W = W;
  I->channels = channels;
  return VF_OK;
}

// Forward (and, with targets, backward into g->grad) over a batch.
vf_status run_train(vf_gate* g, const Images& I, const uint8_t* targets, cudaStream_t s,
                    float* d_loss, float* d_prob) {
  const long long P = (long long)I.count * I.H * I.W;
  vf_status st = ensure_scratch(g, P);
  if (st != VF_OK) return st;
  const int blocks = (int)((P + kThreads - 1) / kThreads);
  conv_fwd<3, kC, true><<<blocks, kThreads, 0, s>>>(I, g->wb, OFF_W1, OFF_B1, nullptr, g->z1);
  conv_fwd<kC, kC, false><<<blocks, kThreads, 0, s>>>(I, g->wb, OFF_W2, OFF_B2, g->z1, g->z2);
  conv_fwd<kC, 1, false><<<blocks, kThreads, 0, s>>>(I, g->wb, OFF_W3, OFF_B3, g->z2, g->z3);
  float* dz3 = g->dz1;  // reused: dz3 has one channel
  bce_head<<<blocks, kThreads, 0, s>>>(I, g->z3, targets, dz3, d_prob, g->loss_part);
  if (targets) {
    if (d_loss) sum_partials<<<1, kThreads, 0, s>>>(g->loss_part, blocks, 1.0f / (float)P, d_loss);
    cudaMemsetAsync(g->part, 0, sizeof(float) * (size_t)kWgradBlocks * NPARAM, s);
    conv_wgrad<kC, 1, false><<<dim3(kWgradBlocks, kC), kThreads, 0, s>>>(I, g->z2, dz3, OFF_W3,
                                                                          OFF_B3, g->part);
    conv_igrad<kC, 1><<<blocks, kThreads, 0, s>>>(I, g->wb, OFF_W3, dz3, g->z2, g->dz2);
    conv_wgrad<kC, kC, false><<<dim3(kWgradBlocks, kC * kC), kThreads, 0, s>>>(
        I, g->z1, g->dz2, OFF_W2, OFF_B2, g->part);
    conv_igrad<kC, kC><<<blocks, kThreads, 0, s>>>(I, g->wb, OFF_W2, g->dz2, g->z1, g->dz1);
    conv_wgrad<3, kC, true><<<dim3(kWgradBlocks, 3 * kC), kThreads, 0, s>>>(I, nullptr, g->dz1,
                                                                            OFF_W1, OFF_B1, g->part);
    reduce_grads<<<(NPARAM + 255) / 256, 256, 0, s>>>(g->part, kWgradBlocks, g->grad);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(g->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  return VF_OK;
}


// Sparse form of the gated filter, first kernel: every unflagged pixel is
// copied and every flagged one listed (y * width + x).  A CTA takes 1,024
// pixels at a time (four per thread, each group of 256 coalesced), counts
// its flagged ones with warp ballots and claims their list slots with one
// atomic add; the order of the list varies between runs (a listed pixel's
// output does not depend on it).  Once the list is longer than `limit` the
// tile form will run and rewrite every pixel, so the CTA stops.
constexpr int kCompactPer = 4;  // pixels per thread and round
__global__ void __launch_bounds__(256)
    gated_compact(const __grid_constant__ Launch L, const uint8_t* __restrict__ flags,
                  long long flag_pitch, int* __restrict__ list, unsigned* __restrict__ count,
                  unsigned limit) {
  __shared__ unsigned s_off[8];  // per warp: first slot after the CTA's base
  __shared__ unsigned s_base, s_tot;
  const long long total = (long long)L.width * L.height;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const long long chunk = 256LL * kCompactPer, step = (long long)gridDim.x * chunk;
  for (long long c0 = blockIdx.x * chunk; c0 < total; c0 += step) {  // uniform over the CTA
    unsigned m[kCompactPer];
    unsigned mine = 0;
#pragma unroll
    for (int k = 0; k < kCompactPer; ++k) {
      const long long i = c0 + k * 256 + threadIdx.x;
      bool f = false;
      if (i < total) {
        const int y = (int)(i / L.width), x = (int)(i - (long long)y * L.width);
        f = flags[(long long)y * flag_pitch + x] != 0;
        if (!f) store_px(L, x, y, load_px(L, x, y));
      }
      m[k] = __ballot_sync(0xffffffffu, f);
      mine += __popc(m[k]);
    }
    if (lane == 0) s_off[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned tot = 0;
      for (int w = 0; w < 8; ++w) {
        const unsigned c = s_off[w];
        s_off[w] = tot;
        tot += c;
      }
      s_tot = tot;
      s_base = tot ? atomicAdd(count, tot) : 0u;
    }
    __syncthreads();
    const unsigned base = s_base, tot = s_tot;
    if (tot != 0u && base + tot > limit) return;  // uniform: the tile form takes the call
    unsigned slot = base + s_off[warp];
#pragma unroll
    for (int k = 0; k < kCompactPer; ++k) {
      if ((m[k] >> lane) & 1u) list[slot + __popc(m[k] & below)] = (int)(c0 + k * 256 + threadIdx.x);
      slot += __popc(m[k]);
    }
    __syncthreads();  // s_off and s_base are rewritten in the next round
  }
}

}  // namespace

extern "C" {

vf_status vf_gate_create(vf_ctx* ctx, unsigned long long seed, vf_gate** out) {
  if (!ctx || !out) return VF_ERR_ARG;
  *out = nullptr;
  vf_gate* g = alloc_refused() ? nullptr : new (std::nothrow) vf_gate();
  if (!g) return VF_ERR_OOM;
  g->ctx = ctx;
  g->seed = seed;
  cudaError_t e = device_alloc(&g->theta, NPARAM * 4);
  if (e == cudaSuccess) e = device_alloc(&g->m, NPARAM * 4);
  if (e == cudaSuccess) e = device_alloc(&g->v, NPARAM * 4);
  if (e == cudaSuccess) e = device_alloc(&g->grad, NPARAM * 4);
  if (e == cudaSuccess) e = device_alloc(&g->wb, NPARAM * 2);
  if (e == cudaSuccess) e = device_alloc(&g->part, sizeof(float) * (size_t)kWgradBlocks * NPARAM);
  if (e == cudaSuccess) e = device_alloc(&g->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(g->d_status, 0, sizeof(int));
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    vf_gate_destroy(g);
    return set_error(ctx, VF_ERR_OOM, "gate allocation failed");
  }
  // He-normal initial weights from a counter-based generator (splitmix64 +
  // Box-Muller), zero biases
  std::vector<float> h(NPARAM, 0.0f);
  auto mix = [](unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto uni = [&](unsigned long long k) {
    return ((mix(seed * 0x100000001B3ull + k) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](int off, int n, int fan_in) {
    for (int k = 0; k < n; ++k) {
      double u1 = uni(2ull * (off + k)), u2 = uni(2ull * (off + k) + 1);
      double nrm = std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
      h[off + k] = (float)(nrm * std::sqrt(2.0 / fan_in));
    }
  };
  fill(OFF_W1, 432, 27);
  fill(OFF_W2, 2304, 144);
  fill(OFF_W3, 144, 144);
  vf_status st = vf_gate_set_params(g, h.data(), NPARAM);
  if (st != VF_OK) {
    vf_gate_destroy(g);
    return st;
  }
  *out = g;
  return VF_OK;
}

vf_status vf_gate_set_params(vf_gate* g, const float* params, int n) {
  if (!g || !params || n != NPARAM) return VF_ERR_ARG;
  cudaError_t e = cudaMemcpy(g->theta, params, NPARAM * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(g->m, 0, NPARAM * 4);
  if (e == cudaSuccess) e = cudaMemset(g->v, 0, NPARAM * 4);
  if (e == cudaSuccess) {
    to_bf16<<<(NPARAM + 255) / 256, 256>>>(g->theta, g->wb);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return set_error(g->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  g->step = 0;
  return VF_OK;
}

vf_status vf_gate_get_params(vf_gate* g, float* params, int n) {
  if (!g || !params || n != NPARAM) return VF_ERR_ARG;
  cudaError_t e = cudaMemcpy(params, g->theta, NPARAM * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_error(g->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  return VF_OK;
}

vf_status vf_gate_gradient(vf_gate* g, const uint8_t* d_imgs, const uint8_t* d_targets, int count,
                           int height, int width, int channels, size_t pitch, float* d_grad,
                           float* d_loss, float* d_prob, void* stream) {
  if (!g || !d_targets) return VF_ERR_ARG;
  Images I;
  vf_status st = check_images(g, d_imgs, count, height, width, channels, pitch, &I);
  if (st != VF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  st = run_train(g, I, d_targets, s, d_loss, d_prob);
  if (st != VF_OK) return st;
  if (d_grad) {
    cudaError_t e = cudaMemcpyAsync(d_grad, g->grad, NPARAM * 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return set_error(g->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  }
  return VF_OK;
}

vf_status vf_gate_train_step(vf_gate* g, const uint8_t* d_imgs, const uint8_t* d_targets,
                             int count, int height, int width, int channels, size_t pitch,
                             float lr, float* d_loss, void* stream) {
  if (!g || !d_targets || !(lr > 0.0f)) return VF_ERR_ARG;
  Images I;
  vf_status st = check_images(g, d_imgs, count, height, width, channels, pitch, &I);
  if (st != VF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  st = run_train(g, I, d_targets, s, d_loss, nullptr);
  if (st != VF_OK) return st;
  g->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - (float)std::pow((double)b1, (double)g->step);
  const float c2 = 1.0f - (float)std::pow((double)b2, (double)g->step);
  adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(g->theta, g->m, g->v, g->grad, g->wb, lr, b1, b2,
                                            1e-8f, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(g->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  return VF_OK;
}

vf_status vf_gate_infer(vf_gate* g, const uint8_t* d_in, int height, int width, int channels,
                        size_t pitch, float threshold, uint8_t* d_flags, size_t flag_pitch,
                        float* d_prob, void* stream) {
  if (!g) return VF_ERR_ARG;
  if (!d_flags && !d_prob) return set_error(g->ctx, VF_ERR_ARG, "no output");
  if (!(threshold > 0.0f && threshold < 1.0f))
    return set_error(g->ctx, VF_ERR_ARG, "threshold must be in (0, 1)");
  if (d_flags && flag_pitch < (size_t)width) return set_error(g->ctx, VF_ERR_ARG, "flag pitch");
  Images I;
  vf_status st = check_images(g, d_in, 1, height, width, channels, pitch, &I);
  if (st != VF_OK) return st;
  const float thr = std::log(threshold / (1.0f - threshold));
  cudaError_t e = cudaSuccess;
  const int engine = gate_tensor_cores(g->ctx);
  if (engine == 1) {
    const int tiles_x = (width + G5_X - 1) / G5_X, tiles_y = (height + G5_Y - 1) / G5_Y;
    const long long ntiles = (long long)tiles_x * tiles_y;
    if (ntiles > 0x7fffffffLL) return set_error(g->ctx, VF_ERR_UNSUPPORTED, "image too large");
    const int grid = (int)std::min<long long>(ntiles, 2LL * std::max(g->sms, 1));
    e = cudaFuncSetAttribute(gate_infer_tc5, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G5_SMEM);
    if (e == cudaSuccess) {
      gate_infer_tc5<<<grid, G5_BLOCK, G5_SMEM, (cudaStream_t)stream>>>(
          I, g->wb, thr, d_flags, (long long)flag_pitch, d_prob, tiles_x, (int)ntiles,
          g->d_status);
      e = cudaGetLastError();
    }
  } else if (engine == 2) {
    const int tiles_x = (width + TX - 1) / TX, tiles_y = (height + TY - 1) / TY;
    e = cudaFuncSetAttribute(gate_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TC_SMEM);
    if (e == cudaSuccess) {
      gate_infer_tc<<<tiles_x * tiles_y, TC_THREADS, TC_SMEM, (cudaStream_t)stream>>>(
          I, g->wb, thr, d_flags, (long long)flag_pitch, d_prob, tiles_x);
      e = cudaGetLastError();
    }
  } else {
    const int tiles_x = (width + IX - 1) / IX, tiles_y = (height + IY - 1) / IY;
    static_assert(kInferSmem <= 200 * 1024, "inference tile fits in shared memory");
    e = cudaFuncSetAttribute(gate_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kInferSmem);
    if (e == cudaSuccess) {
      gate_infer<<<tiles_x * tiles_y, IX * IY, kInferSmem, (cudaStream_t)stream>>>(
          I, g->wb, thr, d_flags, (long long)flag_pitch, d_prob, tiles_x);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) return set_error(g->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  return VF_OK;
}

vf_status vf_filter_gated(vf_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int height, int width,
                          int channels, size_t in_pitch, size_t out_pitch, const uint8_t* d_flags,
                          size_t flag_pitch, const vf_params* p, void* stream,
                          unsigned long long* d_stats) {
  if (!ctx) return VF_ERR_ARG;
  if (!d_flags || flag_pitch < (size_t)width) return set_error(ctx, VF_ERR_ARG, "bad flags");
  Launch L;
  LaunchClass cls;
  vf_status st = prepare_launch(ctx, d_in, d_out, height, width, channels, in_pitch, out_pitch, p,
                                d_stats, &L, &cls);
  if (st != VF_OK) return st;
  if (cls.crit == kEVMF || cls.crit == kEVBDF || cls.precision != VF_FP32)
    return set_error(ctx, VF_ERR_UNSUPPORTED, "the gated form runs VMF, BVDF and AMNF in FP32");
  cudaStream_t s = (cudaStream_t)stream;
  // the sparse form (VF_OPT_GATED_SPARSE): compaction, then one window per
  // listed pixel if the list is short enough; the tile form below then
  // returns at once (the choice is read on the device, from the counter)
  const int permille = gated_sparse_permille(ctx);
  const long long total = (long long)width * height;
  if (permille > 0 && total <= 0x7fffffffLL) {
    int* list = nullptr;
    unsigned* count = nullptr;
    st = gated_scratch(ctx, (size_t)total, &list, &count);
    if (st != VF_OK) return st;
    const unsigned limit =
        permille >= 1000 ? 0xffffffffu : (unsigned)(total * permille / 1000);
    int dev = 0, sms = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
      const long long blocks =
          std::min<long long>((total + 256 * kCompactPer - 1) / (256 * kCompactPer), 8LL * sms);
      gated_compact<<<(int)blocks, 256, 0, s>>>(L, d_flags, (long long)flag_pitch, list, count,
                                                limit);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      switch (cls.w) {
        case 3: e = launch_sparse_w3(L, list, count, limit, sms, cls.crit, cls.apx, cls.deg, s); break;
        case 5: e = launch_sparse_w5(L, list, count, limit, sms, cls.crit, cls.apx, cls.deg, s); break;
        default: e = launch_sparse_w7(L, list, count, limit, sms, cls.crit, cls.apx, cls.deg, s); break;
      }
    }
    if (e != cudaSuccess) return set_error(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
    if (permille >= 1000) return VF_OK;
    L.gate_count = count;
    L.gate_limit = limit;
  }
  if (use_pair_reuse(ctx, cls.w, cls.crit)) {
    // the pair-reuse tiles with the flags read in the finish phase (and
    // whole tiles without a flag copied): every pair term of a tile is
    // computed once, which for the angle terms costs less than the
    // per-window loop on the flagged pixels alone
    L.flags = d_flags;
    L.flag_pitch = (long long)flag_pitch;
    L.tiles_x = (width + kTX - 1) / kTX;
    const int rows = reuse_tile_rows(cls.w, cls.crit);
    const long long rgrid = (long long)L.tiles_x * ((height + rows - 1) / rows);
    if (rgrid > 0x7fffffffLL) return set_error(ctx, VF_ERR_UNSUPPORTED, "image too large");
    cudaError_t e = launch_reuse(L, cls.crit, cls.w, cls.apx, cls.deg, (int)rgrid, s);
    if (e != cudaSuccess) return set_error(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
    return VF_OK;
  }
  const int ty = 4;
  L.tiles_x = (width + kTX - 1) / kTX;
  const long long grid = (long long)L.tiles_x * ((height + ty - 1) / ty);
  if (grid > 0x7fffffffLL) return set_error(ctx, VF_ERR_UNSUPPORTED, "image too large");
  cudaError_t e;
  switch (cls.w) {
    case 3: e = launch_gated_w3(L, d_flags, (long long)flag_pitch, cls.crit, cls.apx, cls.deg, ty, (int)grid, s); break;
    case 5: e = launch_gated_w5(L, d_flags, (long long)flag_pitch, cls.crit, cls.apx, cls.deg, ty, (int)grid, s); break;
    default: e = launch_gated_w7(L, d_flags, (long long)flag_pitch, cls.crit, cls.apx, cls.deg, ty, (int)grid, s); break;
  }
  if (e != cudaSuccess) return set_error(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  return VF_OK;
}

vf_status vf_gate_save(vf_gate* g, const char* path) {
  if (!g || !path) return VF_ERR_ARG;
  std::vector<float> buf(3 * NPARAM);
  cudaError_t e = cudaMemcpy(buf.data(), g->theta, NPARAM * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(buf.data() + NPARAM, g->m, NPARAM * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(buf.data() + 2 * NPARAM, g->v, NPARAM * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_error(g->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  std::vector<unsigned char> out;
  auto put = [&](const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    out.insert(out.end(), c, c + n);
  };
  const char magic[8] = {'V', 'F', 'G', 'A', 'T', 'E', '0', '1'};
  const uint32_t version = 1, n = NPARAM;
  put(magic, 8);
  put(&version, 4);
  put(&n, 4);
  put(&g->step, 8);
  put(&g->seed, 8);
  put(buf.data(), buf.size() * 4);
  const uint32_t crc = crc32(out.data(), out.size());
  put(&crc, 4);
  FILE* f = std::fopen(path, "wb");
  if (!f) return set_error(g->ctx, VF_ERR_ARG, "cannot open checkpoint for writing");
  const size_t w = std::fwrite(out.data(), 1, out.size(), f);
  const int rc = std::fclose(f);
  if (w != out.size() || rc != 0) return set_error(g->ctx, VF_ERR_ARG, "checkpoint write failed");
  return VF_OK;
}

vf_status vf_gate_load(vf_gate* g, const char* path) {
  if (!g || !path) return VF_ERR_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return set_error(g->ctx, VF_ERR_ARG, "cannot open checkpoint");
  std::vector<unsigned char> in;
  unsigned char chunk[65536];
  size_t r;
  while ((r = std::fread(chunk, 1, sizeof(chunk), f)) > 0) in.insert(in.end(), chunk, chunk + r);
  std::fclose(f);
  const size_t expect = 8 + 4 + 4 + 8 + 8 + (size_t)3 * NPARAM * 4 + 4;
  if (in.size() != expect || std::memcmp(in.data(), "VFGATE01", 8) != 0)
    return set_error(g->ctx, VF_ERR_ARG, "not a gate checkpoint");
  uint32_t version, n, crc;
  std::memcpy(&version, in.data() + 8, 4);
  std::memcpy(&n, in.data() + 12, 4);
  std::memcpy(&crc, in.data() + expect - 4, 4);
  if (version != 1 || n != NPARAM) return set_error(g->ctx, VF_ERR_ARG, "checkpoint version");
  if (crc32(in.data(), expect - 4) != crc) return set_error(g->ctx, VF_ERR_ARG, "checkpoint CRC");
  unsigned long long step, seed;
  std::memcpy(&step, in.data() + 16, 8);
  std::memcpy(&seed, in.data() + 24, 8);
  const float* buf = (const float*)(in.data() + 32);
  cudaError_t e = cudaMemcpy(g->theta, buf, NPARAM * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->m, buf + NPARAM, NPARAM * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->v, buf + 2 * NPARAM, NPARAM * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    to_bf16<<<(NPARAM + 255) / 256, 256>>>(g->theta, g->wb);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return set_error(g->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  g->step = step;
  g->seed = seed;
  return VF_OK;
}

unsigned long long vf_gate_step_count(const vf_gate* g) { return g ? g->step : 0; }

vf_status vf_gate_check(vf_gate* g) {
  if (!g) return VF_ERR_ARG;
  int st = 0;
  cudaError_t e = cudaMemcpy(&st, g->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && st != 0) e = cudaMemset(g->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return set_error(g->ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  return st ? set_error(g->ctx, VF_ERR_TIMEOUT, "a tensor-core wait of the gate inference gave up")
            : VF_OK;
}

void vf_gate_destroy(vf_gate* g) {
  if (!g) return;
  free_scratch(g);
  for (void* p : {(void*)g->theta, (void*)g->m, (void*)g->v, (void*)g->grad, (void*)g->wb,
                  (void*)g->part, (void*)g->d_status})
    if (p) cudaFree(p);
  delete g;
}

}  // extern "C"
