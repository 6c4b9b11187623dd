// vf_packed.cuh -- packed-precision (FP16x2 / BF16x2) variants of the window
// kernels: the pairwise terms (and the arccos polynomials) run on packed
// two-lane values, the aggregates are accumulated in FP32.
//
// Layout: one CTA covers 64 x TY output pixels; thread t owns the two
// horizontally adjacent outputs (2t, 2t+1) of its row, so lane .x of every
// packed value belongs to the left window and lane .y to the right one.  The
// staged tile is kept as FP32 float4 (as in the FP32 path, for the
// per-sample work) and, in addition, as packed cells cell(c) = (x[c], x[c+1])
// split into even and odd columns, so that sample i of both windows is one
// cell and a warp reads consecutive cells (no bank conflicts).
//
// Scaling: colour values are multiplied by 1/16 before packing for the L2 and
// angle terms (exact in both formats: 8 significant bits), which keeps the
// squared distances of FP16 below its 65504 limit.  The L1 term of AMNF is
// packed unscaled (integers up to 765: exact in FP16, rounded in BF16).
//
// BVDF: dot product, cosine and both polynomials are packed; for z >= 0.5 the
// argument tau = sqrt(1 - z) is formed in FP32 from the exact integer cross
// product (as in the FP32 path), because 1 - z of a packed cosine would lose
// most of its bits near z = 1.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "vf_kernels.cuh"

namespace vf {

constexpr int kPX = 64;  // output columns per packed tile

template <class T>
struct alignas(16) PCell {
  T r, g, b, s;  // s: 16/|x| for BVDF
};

template <class T>
__device__ __forceinline__ T pk2(float a, float b);
template <>
__device__ __forceinline__ __half2 pk2<__half2>(float a, float b) {
  return __floats2half2_rn(a, b);
}
template <>
__device__ __forceinline__ __nv_bfloat162 pk2<__nv_bfloat162>(float a, float b) {
  return __floats2bfloat162_rn(a, b);
}
__device__ __forceinline__ float2 unpk(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ float2 unpk(__nv_bfloat162 v) { return __bfloat1622float2(v); }

// Horner on packed values with FP32 coefficients rounded to the format.
template <int LEN, class T>
__device__ __forceinline__ T horner_pk(const T* c, T z) {
  T acc = c[LEN - 1];
#pragma unroll
  for (int k = LEN - 2; k >= 0; --k) acc = __hfma2(acc, z, c[k]);
  return acc;
}

template <class T>
struct PTermL2 {
  __device__ __forceinline__ float2 operator()(const PCell<T>& a, const PCell<T>& b, float4,
                                               float4, float4, float4) const {
    T dx = __hsub2(a.r, b.r), dy = __hsub2(a.g, b.g), dz = __hsub2(a.b, b.b);
    return unpk(h2sqrt(__hfma2(dx, dx, __hfma2(dy, dy, __hmul2(dz, dz)))));
  }
};

template <class T>
struct PTermL1 {
  __device__ __forceinline__ float2 operator()(const PCell<T>& a, const PCell<T>& b, float4,
                                               float4, float4, float4) const {
    T d = __hadd2(__habs2(__hsub2(a.r, b.r)),
                  __hadd2(__habs2(__hsub2(a.g, b.g)), __habs2(__hsub2(a.b, b.b))));
    return unpk(d);
  }
};

template <class T, int DEG>
struct PTermAngle {
  T lo[DEG + 1], hi[DEG + 1];
  __device__ __forceinline__ PTermAngle(const float* l, const float* h) {
#pragma unroll
    for (int k = 0; k <= DEG; ++k) {
      lo[k] = pk2<T>(l[k], l[k]);
      hi[k] = pk2<T>(h[k], h[k]);
    }
  }
  // fa*, fb*: FP32 samples of the left (A) and right (B) windows
  __device__ __forceinline__ float2 operator()(const PCell<T>& a, const PCell<T>& b, float4 fai,
                                               float4 faj, float4 fbi, float4 fbj) const {
    T dot = __hfma2(a.r, b.r, __hfma2(a.g, b.g, __hmul2(a.b, b.b)));
    T z = __hmin2(__hmul2(dot, __hmul2(a.s, b.s)), pk2<T>(1.0f, 1.0f));
    float2 zf = unpk(z);
    float2 plo = unpk(horner_pk<DEG + 1>(lo, z));
    // FP32 range reduction: tau^2 = |a x b|^2 / (|a|^2 |b|^2 (1 + z))
    float rA = fai.w * faj.w, rB = fbi.w * fbj.w;
    float tA = cross2(fai, faj) * (rA * rA) * rcp_approx(1.0f + zf.x);
    float tB = cross2(fbi, fbj) * (rB * rB) * rcp_approx(1.0f + zf.y);
    float2 phi = unpk(horner_pk<DEG + 1>(hi, pk2<T>(sqrt_approx(tA), sqrt_approx(tB))));
    return make_float2(zf.x < 0.5f ? plo.x : phi.x, zf.y < 0.5f ? plo.y : phi.y);
  }
};

template <class T>
struct PackedSmem {
  float4* px;     // (64 + w) x sh FP32 samples
  uint32_t* raw;  // (64 + w) x sh packed pixels
  PCell<T>* ev;   // sh x cw cells of even columns
  PCell<T>* od;   // sh x cw cells of odd columns
  float2* agg;    // n x threads aggregate slots (lane .x left window, .y right)
  int sw, sh, cw;
};

inline size_t packed_smem_bytes(int w, int ty) {
  size_t sw = kPX + w, sh = ty + w - 1, cw = (kPX + w) / 2 + 1, threads = (size_t)kTX * ty;
  return sw * sh * 20 + 2 * sh * cw * 16 + (size_t)w * w * threads * 8;
}

template <class T>
__device__ __forceinline__ PackedSmem<T> carve_packed(int W, int TY) {
  extern __shared__ __align__(16) unsigned char smem[];
  PackedSmem<T> t;
  t.sw = kPX + W;
  t.sh = TY + W - 1;
  t.cw = (kPX + W) / 2 + 1;
  unsigned char* p = smem;
  t.px = reinterpret_cast<float4*>(p);
  p += (size_t)t.sw * t.sh * 16;
  t.ev = reinterpret_cast<PCell<T>*>(p);
  p += (size_t)t.sh * t.cw * 16;
  t.od = reinterpret_cast<PCell<T>*>(p);
  p += (size_t)t.sh * t.cw * 16;
  t.agg = reinterpret_cast<float2*>(p);
  p += (size_t)W * W * blockDim.x * 8;
  t.raw = reinterpret_cast<uint32_t*>(p);
  return t;
}

// Cell of window sample column i (0..w-1) of thread column tx, row r.
template <class T>
__device__ __forceinline__ const PCell<T>& cell(const PackedSmem<T>& t, int r, int tx, int i) {
  return (i & 1) ? t.od[r * t.cw + tx + (i >> 1)] : t.ev[r * t.cw + tx + (i >> 1)];
}

// Rolled row-pair loop over the two windows of thread column tx, row py;
// aggregates into the thread's float2 slots sagg[i * stride].
template <int W, bool NEED_F32, class T, class Term>
__device__ __forceinline__ void packed_aggregates(const PackedSmem<T>& t, int tx, int py,
                                                  const Term& term, float2* sagg, int stride) {
#pragma unroll
  for (int i = 0; i < W * W; ++i) sagg[i * stride] = make_float2(0.0f, 0.0f);
  const int c0 = 2 * tx;  // left window's first FP32 column
#pragma unroll 1
  for (int a = 0; a < W; ++a) {
    PCell<T> A[W];
    float4 FA[W + 1];
    float2 ra[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      A[i] = cell(t, py + a, tx, i);
      ra[i] = make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int i = 0; i <= W; ++i) FA[i] = NEED_F32 ? t.px[(py + a) * t.sw + c0 + i] : float4{};
#pragma unroll
    for (int i = 0; i < W; ++i)
#pragma unroll
      for (int j = i + 1; j < W; ++j) {
        float2 d = term(A[i], A[j], FA[i], FA[j], FA[i + 1], FA[j + 1]);
        ra[i].x += d.x;
        ra[i].y += d.y;
        ra[j].x += d.x;
        ra[j].y += d.y;
      }
#pragma unroll 1
    for (int b = a + 1; b < W; ++b) {
      PCell<T> B[W];
      float4 FB[W + 1];
      float2 rb[W];
#pragma unroll
      for (int j = 0; j < W; ++j) {
        B[j] = cell(t, py + b, tx, j);
        rb[j] = make_float2(0.0f, 0.0f);
      }
#pragma unroll
      for (int j = 0; j <= W; ++j) FB[j] = NEED_F32 ? t.px[(py + b) * t.sw + c0 + j] : float4{};
#pragma unroll
      for (int i = 0; i < W; ++i)
#pragma unroll
        for (int j = 0; j < W; ++j) {
          float2 d = term(A[i], B[j], FA[i], FB[j], FA[i + 1], FB[j + 1]);
          ra[i].x += d.x;
          ra[i].y += d.y;
          rb[j].x += d.x;
          rb[j].y += d.y;
        }
#pragma unroll
      for (int j = 0; j < W; ++j) {
        float2 v = sagg[(b * W + j) * stride];
        sagg[(b * W + j) * stride] = make_float2(v.x + rb[j].x, v.y + rb[j].y);
      }
    }
#pragma unroll
    for (int i = 0; i < W; ++i) {
      float2 v = sagg[(a * W + i) * stride];
      sagg[(a * W + i) * stride] = make_float2(v.x + ra[i].x, v.y + ra[i].y);
    }
  }
}

// argmin of lane `lane` (0 left, 1 right) over the slots; near-tie test as in
// the FP32 path against FP32 samples of that window (column c0 + lane).
template <int W>
__device__ __forceinline__ Selection packed_select(const float2* sagg, int stride,
                                                   const float4* px, int sw, int c0, int py,
                                                   int lane, bool want_tie) {
  constexpr int N = W * W;
  int best = 0;
  float bv = lane ? sagg[0].y : sagg[0].x;
#pragma unroll
  for (int i = 1; i < N; ++i) {
    float v = lane ? sagg[i * stride].y : sagg[i * stride].x;
    if (v < bv) {
      bv = v;
      best = i;
    }
  }
  Selection s{best, false};
  if (want_tie) {
    const int cx = c0 + lane;
    float4 xb = px[(py + best / W) * sw + cx + best % W];
    float second = __int_as_float(0x7f800000);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float4 xi = px[(py + i / W) * sw + cx + i % W];
      float v = lane ? sagg[i * stride].y : sagg[i * stride].x;
      bool diff = xi.x != xb.x || xi.y != xb.y || xi.z != xb.z;
      if (diff && v < second) second = v;
    }
    s.near_tie = second <= bv * (1.0f + 1e-5f);
  }
  return s;
}

// AMNF weighted mean of one window (left column cx) from its aggregates.
template <int W, int CRIT, int APX, int DEG>
__device__ __forceinline__ uint32_t packed_amnf_finish(const Launch& L, const float4* px,
                                                       const uint32_t* raw, int sw, int cx,
                                                       int py, const float2* sagg, int stride,
                                                       int lane, bool& tie) {
  constexpr int N = W * W, C = N / 2;
  const float4 xc = px[(py + W / 2) * sw + cx + W / 2];
  const uint32_t rawc = raw[(py + W / 2) * sw + cx + W / 2];
  const float aggC = lane ? sagg[C * stride].y : sagg[C * stride].x;
  tie = false;
  if (aggC == 0.0f) return rawc;  // constant window
  float wsum = 0.0f, ax = 0.0f, ay = 0.0f, az = 0.0f;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float4 xi = px[(py + i / W) * sw + cx + i % W];
    float ai = lane ? sagg[i * stride].y : sagg[i * stride].x;
    float rh = rcp_approx(L.kappa_scale * ai);
    float dx = xc.x - xi.x, dy = xc.y - xi.y, dz = xc.z - xi.z;
    float u;
    if constexpr (CRIT == kAMNFE) {
      u = (fabsf(dx) + fabsf(dy) + fabsf(dz)) * rh;
    } else {
      u = 0.5f * fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * (rh * rh);
    }
    float wi = (rh * rh * rh) * expneg<APX, DEG>(L, u);
    wsum += wi;
    ax = fmaf(wi, xi.x, ax);
    ay = fmaf(wi, xi.y, ay);
    az = fmaf(wi, xi.z, az);
  }
  float rw = 1.0f / wsum;
  float yx = ax * rw, yy = ay * rw, yz = az * rw;
  if (L.stats) {
    auto g = [](float v) { return fabsf(v - floorf(v) - 0.5f); };
    tie = fminf(g(yx), fminf(g(yy), g(yz))) < 1e-3f;
  }
  return pack_rgb(round_u8(yx), round_u8(yy), round_u8(yz), rawc);
}

template <int W, int CRIT, int APX, int DEG, class T>
__global__ void __launch_bounds__(256) packed_kernel(const __grid_constant__ Launch L) {
  pdl_begin();
  constexpr int R = W / 2;
  const int TY = blockDim.x / kTX;
  const PackedSmem<T> t = carve_packed<T>(W, TY);
  const int tile = blockIdx.x;
  const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
  const int x0 = txi * kPX, y0 = tyi * TY;
  // scale of the packed colours: 1/16 for L2 and angles, 1 for L1
  const float S = (CRIT == kAMNFE || CRIT == kAMNFG) ? 1.0f : 0.0625f;

  // FP32 samples and packed pixels of the (64 + w) x (TY + w - 1) region
  const int cells = t.sw * t.sh;
  for (int idx = threadIdx.x; idx < cells; idx += blockDim.x) {
    int ry = idx / t.sw, rx = idx - ry * t.sw;
    int gy = min(max(y0 + ry - R, 0), L.height - 1);
    int gx = min(max(x0 + rx - R, 0), L.width - 1);
    uint32_t v = load_px(L, gx, gy);
    float r = (float)(v & 255u), g = (float)((v >> 8) & 255u), b = (float)((v >> 16) & 255u);
    float w = 0.0f;
    if (CRIT == kBVDF) {
      float n2 = fmaf(r, r, fmaf(g, g, b * b));
      if (n2 > 0.0f) {
        float y = rsqrtf(n2);
        w = y * fmaf(-0.5f * n2 * y, y, 1.5f);
      }
    }
    t.px[idx] = make_float4(r, g, b, w);
    t.raw[idx] = v;
  }
  __syncthreads();
  // packed cells: cell(c) = (x[c], x[c+1]) for c = 0 .. 64 + w - 2
  const int ncell = t.sw - 1;
  for (int idx = threadIdx.x; idx < t.sh * ncell; idx += blockDim.x) {
    int ry = idx / ncell, c = idx - ry * ncell;
    float4 p = t.px[ry * t.sw + c], q = t.px[ry * t.sw + c + 1];
    PCell<T> cl;
    cl.r = pk2<T>(p.x * S, q.x * S);
    cl.g = pk2<T>(p.y * S, q.y * S);
    cl.b = pk2<T>(p.z * S, q.z * S);
    cl.s = pk2<T>(p.w * 16.0f, q.w * 16.0f);
    if (c & 1) t.od[ry * t.cw + (c >> 1)] = cl;
    else t.ev[ry * t.cw + (c >> 1)] = cl;
  }
  __syncthreads();

  const int tx = threadIdx.x % kTX, py = threadIdx.x / kTX;
  const int c0 = 2 * tx;
  const int gy = y0 + py;
  const bool want_tie = L.stats != nullptr;
  float2* sagg = t.agg + threadIdx.x;
  const int stride = blockDim.x;
  int ties = 0, switched = 0, pixels = 0;

  bool run_pairs = true, sw[2] = {false, false};
  if constexpr (CRIT == kEVMF) {
    // switch of both windows in FP32 (vf_kernels.cuh), pairs only if needed
    TileSmem ts;
    ts.px = t.px;
    ts.raw = t.raw;
    ts.sw = t.sw;
    bool tie0 = false, tie1 = false;
    sw[0] = x0 + c0 < L.width && gy < L.height && evmf_switch<W, APX, DEG>(L, ts, c0, py, tie0);
    sw[1] = x0 + c0 + 1 < L.width && gy < L.height &&
            evmf_switch<W, APX, DEG>(L, ts, c0 + 1, py, tie1);
    ties += tie0 + tie1;
    switched = sw[0] + sw[1];
    run_pairs = sw[0] || sw[1];
  }
  if (run_pairs) {
    if constexpr (CRIT == kBVDF) {
      packed_aggregates<W, true>(t, tx, py, PTermAngle<T, DEG>(L.c.a, L.c.b), sagg, stride);
    } else if constexpr (CRIT == kAMNFE || CRIT == kAMNFG) {
      packed_aggregates<W, false>(t, tx, py, PTermL1<T>{}, sagg, stride);
    } else {
      packed_aggregates<W, false>(t, tx, py, PTermL2<T>{}, sagg, stride);
    }
  }
#pragma unroll
  for (int lane = 0; lane < 2; ++lane) {
    const int gx = x0 + c0 + lane;
    if (gx >= L.width || gy >= L.height) continue;
    ++pixels;
    const int cx = c0 + lane;
    uint32_t v;
    if constexpr (CRIT == kAMNFE || CRIT == kAMNFG) {
      bool tie = false;
      v = packed_amnf_finish<W, CRIT, APX, DEG>(L, t.px, t.raw, t.sw, cx, py, sagg, stride, lane,
                                                tie);
      ties += tie;
    } else {
      if (CRIT == kEVMF && !sw[lane]) {
        v = t.raw[(py + R) * t.sw + cx + R];
      } else {
        Selection s = packed_select<W>(sagg, stride, t.px, t.sw, c0, py, lane, want_tie);
        v = t.raw[(py + s.best / W) * t.sw + cx + s.best % W];
        ties += s.near_tie;
      }
    }
    store_px(L, gx, gy, v);
  }
  block_stats(L, pixels, ties, switched);
}

}  // namespace vf
