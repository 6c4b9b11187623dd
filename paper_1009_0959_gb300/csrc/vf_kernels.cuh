// vf_kernels.cuh -- sm_103a per-window kernels of the sliding-window vector
// filters (Sec. 3: y(r,c) = F(W(r,c))).
//
// One CTA filters a tile of 32 x TY output pixels (32 x 2TY when each thread
// filters two windows).  It stages the tile plus a (w-1)/2 halo into shared
// memory once (coalesced 32-bit RGBX loads, borders replicated): the packed
// pixels, and FP32 colours where a term needs them.  Each thread walks the
// n(n-1)/2 pairs of its window, each pairwise term computed once and added to
// the aggregates of both samples; the L2 and L1 terms are formed on the
// packed bytes with integer SIMD instructions (exact integers).
//
// Pair loop organisation: the window is processed as blocks of two rows
// (a <= b); a block's samples are held in registers while its w*w (or
// w(w-1)/2) pairs are formed.  For small windows (w = 3, and w = 5 with the
// cheap distance terms) everything is unrolled and the n aggregates live in
// registers; otherwise the row-pair loop stays rolled (keeping the code small
// enough for the instruction cache) and each block's partial sums are added
// to per-thread aggregate slots in shared memory.  VMF and AMNF threads filter
// two vertically adjacent windows and form their shared samples' pairs once
// (process_tile2).  The pair-reuse kernels (vf_reuse.cuh) and the EVMF work
// queue (vf_evmf.cuh) build on the helpers here.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "vf_internal.h"

namespace vf {

// ---------------------------------------------------------------- helpers

// Programmatic dependent launch (sm_90 and later).  A filter kernel launched
// with programmatic stream serialisation may have its CTAs scheduled while
// the previous kernel of the stream drains; griddepcontrol.wait then holds
// them until that kernel has completed and its memory is visible, before
// any device-memory access, so stream order is kept.  Right after, the
// kernel allows its own successor to be scheduled (that one waits the same
// way).  Without the launch attribute both instructions return at once.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch `kern` with the programmatic-serialisation attribute when `pdl`.
template <typename... KArgs, typename... Args>
cudaError_t launch_maybe_pdl(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block,
                             size_t smem, cudaStream_t s, const Args&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Horner evaluation of sum_k c[k] z^k, LEN coefficients.
template <int LEN>
__device__ __forceinline__ float horner(const float* c, float z) {
  float acc = c[LEN - 1];
#pragma unroll
  for (int k = LEN - 2; k >= 0; --k) acc = fmaf(acc, z, c[k]);
  return acc;
}

__device__ __forceinline__ uint32_t load_px(const Launch& L, int gx, int gy) {
  const uint8_t* p = L.in + (long long)gy * L.in_pitch + (long long)gx * L.channels;
  if (L.vec4_in) return *reinterpret_cast<const uint32_t*>(p);
  uint32_t v = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16);
  if (L.channels == 4) v |= (uint32_t)p[3] << 24;
  return v;
}

__device__ __forceinline__ void store_px(const Launch& L, int gx, int gy, uint32_t v) {
  uint8_t* p = L.out + (long long)gy * L.out_pitch + (long long)gx * L.channels;
  if (L.vec4_out) {
    *reinterpret_cast<uint32_t*>(p) = v;
    return;
  }
  p[0] = (uint8_t)v;
  p[1] = (uint8_t)(v >> 8);
  p[2] = (uint8_t)(v >> 16);
  if (L.channels == 4) p[3] = (uint8_t)(v >> 24);
}

// ---------------------------------------------------------------- pairwise terms

// Sec. 3.3 (first branch of Eq. equ_evf): Euclidean distance.  The squared
// distance of two 8-bit colours is an exact integer in FP32.
struct TermL2 {
  __device__ __forceinline__ float operator()(float4 a, float4 b) const {
    float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    return sqrt_approx(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  }
};

// The same distance on packed 8-bit colours (fourth byte zero): __vabsdiffu4
// forms the byte-wise |a_k - b_k| and one __dp4a squares and sums them, the
// exact integer d2 < 2^18.  Accumulated onto the bits of 2^23 it reads as the
// FP32 number 2^23 + d2, and one subtraction leaves d2 exactly: the value the
// FP32 form computes, so the same square root, from two integer-pipe and one
// FP32 instruction instead of six FP32 ones.
struct TermL2U8 {
  __device__ __forceinline__ float operator()(uint32_t a, uint32_t b) const {
    const uint32_t d = __vabsdiffu4(a, b);
    const float d2 = __uint_as_float(__dp4a(d, d, 0x4B000000u)) - 8388608.0f;
    return sqrt_approx(d2);
  }
};

// Sec. 3.2: city-block distance (exact integer in FP32).
struct TermL1 {
  __device__ __forceinline__ float operator()(float4 a, float4 b) const {
    return fabsf(a.x - b.x) + fabsf(a.y - b.y) + fabsf(a.z - b.z);
  }
};

// |a x b|^2 from exact integer components: each component is a difference of
// two products < 2^24, exact in FP32 with one FMA.
__device__ __forceinline__ float cross2(float4 a, float4 b) {
  float cx = fmaf(a.y, b.z, -(a.z * b.y));
  float cy = fmaf(a.z, b.x, -(a.x * b.z));
  float cz = fmaf(a.x, b.y, -(a.y * b.x));
  return fmaf(cx, cx, fmaf(cy, cy, cz * cz));
}

// Sec. 3.1, exact angle A = arccos(a.b / (|a||b|)).  Evaluated through the
// half-angle identity tan(A/2) = |a x b| / (|a||b| + a.b): colour vectors
// are non-negative, so a.b >= 0, A is in [0, pi/2] and u = tan(A/2) is in
// [0, 1) -- the same angle without the loss of arccos near 1, from the exact
// integer cross and dot products.  A = 2 atan(u) = u P(u^2), P the library's
// degree-7 minimax polynomial of 2 atan(sqrt s) / sqrt s on [0, 1] (Remez
// exchange on the host, VF_FN_HALF_ANGLE; relative error 1.1e-7 before FP32
// rounding, about that of a single-precision arctangent): no quadrant cases,
// no divergent branches, FMA chains only.  c = its kHalfAngleCoeffs
// coefficients.  .w holds 1/|x| (0 for the zero vector); a pair with a zero
// vector has angle pi/2.
constexpr int kHalfAngleCoeffs = 8;
struct TermAngleExact {
  const float* c;
  __device__ __forceinline__ explicit TermAngleExact(const float* k) : c(k) {}
  __device__ __forceinline__ float operator()(float4 a, float4 b) const {
    const float dot = fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
    const float s = sqrt_approx(cross2(a, b));
    const float rr = a.w * b.w;  // 1 / (|a||b|)
    const float u = s * rr * rcp_approx(fmaf(dot, rr, 1.0f));  // 1 + cos in [1, 2]
    const float ang = u * horner<kHalfAngleCoeffs>(c, u * u);
    return rr == 0.0f ? 1.57079632679f : ang;
  }
};

// Sec. 3.1, approximate angle: z = cos; z < 0.5: the arccos approximant of
// Table 1 (ARCCOS row); z >= 0.5: tau = sqrt(1 - z) and the approximant of
// 2 arcsin(tau / sqrt 2) (ARCSIN row).  1 - z is formed as
// |a x b|^2 / (|a|^2 |b|^2 (1 + z)) so that tau keeps full relative
// precision for nearly parallel colours.
template <int DEG>
struct TermAngleApprox {
  float lo[DEG + 1];  // coefficients held in registers for the pair loop
  float hi[DEG + 1];
  __device__ __forceinline__ TermAngleApprox(const float* l, const float* h) {
#pragma unroll
    for (int k = 0; k <= DEG; ++k) {
      lo[k] = l[k];
      hi[k] = h[k];
    }
  }
  __device__ __forceinline__ float operator()(float4 a, float4 b) const {
    float dot = fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
    float rr = a.w * b.w;  // 1 / (|a||b|), 0 for a zero vector
    float z = fminf(dot * rr, 1.0f);
    float plo = horner<DEG + 1>(lo, z);
    float t2 = cross2(a, b) * (rr * rr) * rcp_approx(1.0f + z);
    float phi = horner<DEG + 1>(hi, sqrt_approx(t2));
    return z < 0.5f ? plo : phi;
  }
};

// ---------------------------------------------------------------- window aggregates

// A window sample: an FP32 colour (staged .w kept) or a packed 8-bit colour
// with the fourth byte cleared.
__device__ __forceinline__ float4 load_sample(const float4* p) { return *p; }
__device__ __forceinline__ uint32_t load_sample(const uint32_t* p) { return *p & 0x00ffffffu; }
__device__ __forceinline__ bool same_colour(float4 a, float4 b) {
  return a.x == b.x && a.y == b.y && a.z == b.z;
}
__device__ __forceinline__ bool same_colour(uint32_t a, uint32_t b) { return a == b; }

// Per-thread window view: the window of output pixel (px, py) of the tile is
// rows py..py+W-1, columns px..px+W-1 of the staged tile (pitch sw).

// w <= 5: all n aggregates in registers, fully unrolled.
template <int W, class Term, class S>
__device__ __forceinline__ void aggregates_reg(const S* tile, int sw, int px, int py,
                                               const Term& term, float (&agg)[W * W]) {
#pragma unroll
  for (int i = 0; i < W * W; ++i) agg[i] = 0.0f;
#pragma unroll
  for (int a = 0; a < W; ++a) {
    S A[W];
#pragma unroll
    for (int i = 0; i < W; ++i) A[i] = load_sample(tile + (py + a) * sw + px + i);
#pragma unroll
    for (int i = 0; i < W; ++i)
#pragma unroll
      for (int j = i + 1; j < W; ++j) {
        float t = term(A[i], A[j]);
        agg[a * W + i] += t;
        agg[a * W + j] += t;
      }
#pragma unroll
    for (int b = a + 1; b < W; ++b) {
      S B[W];
#pragma unroll
      for (int j = 0; j < W; ++j) B[j] = load_sample(tile + (py + b) * sw + px + j);
#pragma unroll
      for (int i = 0; i < W; ++i)
#pragma unroll
        for (int j = 0; j < W; ++j) {
          float t = term(A[i], B[j]);
          agg[a * W + i] += t;
          agg[b * W + j] += t;
        }
    }
  }
}

// Rolled row-pair loop (w = 7, and w = 5 for the costly angle term); aggregates in shared memory slots
// sagg[i * stride] (stride = threads per CTA, so a warp's slots are
// consecutive words).
template <int W, class Term, class S>
__device__ __forceinline__ void aggregates_smem(const S* tile, int sw, int px, int py,
                                                const Term& term, float* sagg, int stride) {
#pragma unroll
  for (int i = 0; i < W * W; ++i) sagg[i * stride] = 0.0f;
#pragma unroll 1
  for (int a = 0; a < W; ++a) {
    S A[W];
    float ra[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      A[i] = load_sample(tile + (py + a) * sw + px + i);
      ra[i] = 0.0f;
    }
#pragma unroll
    for (int i = 0; i < W; ++i)
#pragma unroll
      for (int j = i + 1; j < W; ++j) {
        float t = term(A[i], A[j]);
        ra[i] += t;
        ra[j] += t;
      }
#pragma unroll 1
    for (int b = a + 1; b < W; ++b) {
      S B[W];
      float rb[W];
#pragma unroll
      for (int j = 0; j < W; ++j) {
        B[j] = load_sample(tile + (py + b) * sw + px + j);
        rb[j] = 0.0f;
      }
#pragma unroll
      for (int i = 0; i < W; ++i)
#pragma unroll
        for (int j = 0; j < W; ++j) {
          float t = term(A[i], B[j]);
          ra[i] += t;
          rb[j] += t;
        }
#pragma unroll
      for (int j = 0; j < W; ++j) sagg[(b * W + j) * stride] += rb[j];
    }
#pragma unroll
    for (int i = 0; i < W; ++i) sagg[(a * W + i) * stride] += ra[i];
  }
}

// argmin_i agg[i], lowest index on an exact tie; optionally the near-tie test
// against the best aggregate of a sample with a different colour.
struct Selection {
  int best;
  bool near_tie;
};

template <int W, bool REG, class S>
__device__ __forceinline__ Selection select_min(const float* agg_reg, const float* sagg, int stride,
                                                const S* tile, int sw, int px, int py,
                                                bool want_tie) {
  constexpr int N = W * W;
  int best = 0;
  float bv = REG ? agg_reg[0] : sagg[0];
#pragma unroll
  for (int i = 1; i < N; ++i) {
    float v = REG ? agg_reg[i] : sagg[i * stride];
    if (v < bv) {
      bv = v;
      best = i;
    }
  }
  Selection s{best, false};
  if (want_tie) {
    const S xb = load_sample(tile + (py + best / W) * sw + px + best % W);
    float second = __int_as_float(0x7f800000);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const S xi = load_sample(tile + (py + i / W) * sw + px + i % W);
      float v = REG ? agg_reg[i] : sagg[i * stride];
      bool diff = !same_colour(xi, xb);
      if (diff && v < second) second = v;
    }
    s.near_tie = second <= bv * (1.0f + 1e-5f);
  }
  return s;
}

// Selection over the window of (px, py) with pairwise term `term`; REG picks
// register aggregates (fully unrolled) or shared-memory slots (rolled).
template <int W, bool REG, class Term, class S>
__device__ __forceinline__ Selection window_select(const S* tile, int sw, int px, int py,
                                                   const Term& term, float* sagg, int stride,
                                                   bool want_tie) {
  if constexpr (REG) {
    float agg[W * W];
    aggregates_reg<W>(tile, sw, px, py, term, agg);
    return select_min<W, true>(agg, nullptr, 0, tile, sw, px, py, want_tie);
  } else {
    aggregates_smem<W>(tile, sw, px, py, term, sagg, stride);
    return select_min<W, false>(nullptr, sagg, stride, tile, sw, px, py, want_tie);
  }
}

// ---------------------------------------------------------------- elementary functions

// Sec. 3.2: exp(-u) with the cut-off (0 outside [0, T]).
template <int APX, int DEG>
__device__ __forceinline__ float expneg(const Launch& L, float u) {
  float e;
  if constexpr (APX == kExact) {
    e = expf(-u);
  } else if constexpr (APX == kPoly) {
    e = horner<DEG + 1>(L.c.a, u);
  } else {
    e = horner<5>(L.c.a, u) * rcp_approx(horner<5>(L.c.b, u));
  }
  return (u > L.exp_cutoff) ? 0.0f : e;
}

// Sec. 3.3: z ln z with the cut-off (0 below T).  ALT: the polynomial of
// the EVBDF switch (L.c.e; a and b hold its arccos pieces).
template <int APX, int DEG, bool ALT = false>
__device__ __forceinline__ float ent(const Launch& L, float z) {
  float e;
  if constexpr (APX == kExact) {
    e = z * logf(z);
  } else if constexpr (APX == kPoly) {
    e = horner<DEG + 1>(ALT ? L.c.e : L.c.a, z);
  } else {
    e = horner<5>(L.c.a, z) * rcp_approx(horner<5>(L.c.b, z));
  }
  return (z < L.ent_cutoff || z <= 0.0f) ? 0.0f : e;
}

// ---------------------------------------------------------------- the kernel

struct TileSmem {
  float4* px;     // SH x SW staged colours (FP32), .w per criterion
  uint32_t* raw;  // SH x SW original packed pixels
  float* agg;     // N x threads aggregate slots (w = 7)
  int* list;      // threads: EVMF compacted pixel list
  int sw, sh;
};

__device__ __forceinline__ TileSmem carve(int W, bool reg, int TY, int threads) {
  extern __shared__ __align__(16) unsigned char smem[];
  TileSmem t;
  t.sw = kTX + W - 1;
  t.sh = TY + W - 1;
  int cells = t.sw * t.sh;
  t.px = reinterpret_cast<float4*>(smem);
  t.raw = reinterpret_cast<uint32_t*>(smem + cells * 16);
  unsigned char* p = smem + cells * 20;
  t.agg = reinterpret_cast<float*>(p);
  if (!reg) p += (size_t)W * W * threads * 4;
  t.list = reinterpret_cast<int*>(p);
  return t;
}

// FLOATS = false stages only the packed pixels (the VMF selection works on
// them directly).
// A staged sample's FP32 colour; .w = 1/|x| for the angle criteria (0 for
// the zero vector), 0 otherwise.
template <int CRIT>
__device__ __forceinline__ float4 stage_cell(uint32_t v) {
  float r = (float)(v & 255u), g = (float)((v >> 8) & 255u), b = (float)((v >> 16) & 255u);
  float w = 0.0f;
  if (CRIT == kBVDF || CRIT == kEVBDF) {
    float n2 = fmaf(r, r, fmaf(g, g, b * b));
    if (n2 > 0.0f) {
      float y = rsqrtf(n2);
      w = y * fmaf(-0.5f * n2 * y, y, 1.5f);  // one Newton step
    }
  }
  return make_float4(r, g, b, w);
}

template <int CRIT, bool FLOATS = true>
__device__ __forceinline__ void stage_tile(const Launch& L, const TileSmem& t, int x0, int y0, int R) {
  const int cells = t.sw * t.sh;
  for (int idx = threadIdx.x; idx < cells; idx += blockDim.x) {
    int ry = idx / t.sw, rx = idx - ry * t.sw;
    int gy = min(max(y0 + ry - R, 0), L.height - 1);
    int gx = min(max(x0 + rx - R, 0), L.width - 1);
    uint32_t v = load_px(L, gx, gy);
    t.raw[idx] = v;
    if constexpr (!FLOATS) continue;
    t.px[idx] = stage_cell<CRIT>(v);
  }
}

__device__ __forceinline__ uint32_t pack_rgb(int r, int g, int b, uint32_t keep) {
  return (uint32_t)r | ((uint32_t)g << 8) | ((uint32_t)b << 16) | (keep & 0xff000000u);
}

__device__ __forceinline__ int round_u8(float v) { return min(max(__float2int_rn(v), 0), 255); }

__device__ __forceinline__ void block_stats(const Launch& L, int pixels, int ties, int switched) {
  if (L.stats == nullptr) return;
  // warp-level reduction, one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pixels += __shfl_xor_sync(0xffffffffu, pixels, o);
    ties += __shfl_xor_sync(0xffffffffu, ties, o);
    switched += __shfl_xor_sync(0xffffffffu, switched, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (pixels) atomicAdd(L.stats + 0, (unsigned long long)pixels);
    if (ties) atomicAdd(L.stats + 1, (unsigned long long)ties);
    if (switched) atomicAdd(L.stats + 2, (unsigned long long)switched);
  }
}

// AMNF (Sec. 3.2, Eq. equ_amnf) of the window of (px, py).
// City-block aggregates sum_j ||x_i - x_j||_1 on the packed 8-bit pixels:
// __vsadu4 sums the absolute differences of the four bytes and adds its
// accumulator in one integer-pipe instruction (the fourth byte is masked to
// 0), so each pair costs two instructions instead of seven FP32 ones.  The
// sums are exact integers (< 2^16), the same values the FP32 path forms.
template <int W>
__device__ __forceinline__ void l1_aggregates_int(const uint32_t* raw, int sw, int px, int py,
                                                  uint32_t (&agg)[W * W]) {
#pragma unroll
  for (int i = 0; i < W * W; ++i) agg[i] = 0u;
#pragma unroll
  for (int a = 0; a < W; ++a) {
    uint32_t A[W];
#pragma unroll
    for (int i = 0; i < W; ++i) A[i] = raw[(py + a) * sw + px + i] & 0x00ffffffu;
#pragma unroll
    for (int i = 0; i < W; ++i)
#pragma unroll
      for (int j = i + 1; j < W; ++j) {
        agg[a * W + i] = __vsadu4(A[i], A[j]) + agg[a * W + i];
        agg[a * W + j] = __vsadu4(A[i], A[j]) + agg[a * W + j];
      }
#pragma unroll
    for (int b = a + 1; b < W; ++b) {
      uint32_t B[W];
#pragma unroll
      for (int j = 0; j < W; ++j) B[j] = raw[(py + b) * sw + px + j] & 0x00ffffffu;
#pragma unroll
      for (int i = 0; i < W; ++i)
#pragma unroll
        for (int j = 0; j < W; ++j) {
          agg[a * W + i] = __vsadu4(A[i], B[j]) + agg[a * W + i];
          agg[b * W + j] = __vsadu4(A[i], B[j]) + agg[b * W + j];
        }
    }
  }
}

// The same with the rolled row-pair loop and per-thread shared-memory slots
// (integers written into the float slots' storage).
template <int W>
__device__ __forceinline__ void l1_aggregates_int_smem(const uint32_t* raw, int sw, int px, int py,
                                                       uint32_t* sagg, int stride) {
#pragma unroll
  for (int i = 0; i < W * W; ++i) sagg[i * stride] = 0u;
#pragma unroll 1
  for (int a = 0; a < W; ++a) {
    uint32_t A[W], ra[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      A[i] = raw[(py + a) * sw + px + i] & 0x00ffffffu;
      ra[i] = 0u;
    }
#pragma unroll
    for (int i = 0; i < W; ++i)
#pragma unroll
      for (int j = i + 1; j < W; ++j) {
        ra[i] = __vsadu4(A[i], A[j]) + ra[i];
        ra[j] = __vsadu4(A[i], A[j]) + ra[j];
      }
#pragma unroll 1
    for (int b = a + 1; b < W; ++b) {
      uint32_t B[W], rb[W];
#pragma unroll
      for (int j = 0; j < W; ++j) {
        B[j] = raw[(py + b) * sw + px + j] & 0x00ffffffu;
        rb[j] = 0u;
      }
#pragma unroll
      for (int i = 0; i < W; ++i)
#pragma unroll
        for (int j = 0; j < W; ++j) {
          ra[i] = __vsadu4(A[i], B[j]) + ra[i];
          rb[j] = __vsadu4(A[i], B[j]) + rb[j];
        }
#pragma unroll
      for (int j = 0; j < W; ++j) sagg[(b * W + j) * stride] += rb[j];
    }
#pragma unroll
    for (int i = 0; i < W; ++i) sagg[(a * W + i) * stride] += ra[i];
  }
#pragma unroll
  for (int i = 0; i < W * W; ++i)
    reinterpret_cast<float*>(sagg)[i * stride] = (float)sagg[i * stride];
}

// AMNF output of the window of (px, py) from its aggregates h_i (agg(i)):
// weights w_i = h_i^-3 K((x_C - x_i) / h_i), weighted mean, rounded.
template <int W, int CRIT, int APX, int DEG, class Agg>
__device__ __forceinline__ uint32_t amnf_finish(const Launch& L, const TileSmem& t, int px, int py,
                                                const Agg& agg, bool& tie) {
  constexpr int N = W * W, C = N / 2;
  const float4 xc = t.px[(py + W / 2) * t.sw + px + W / 2];
  const uint32_t rawc = t.raw[(py + W / 2) * t.sw + px + W / 2];
  if (agg(C) == 0.0f) {  // constant window: every h_i is 0, output the centre
    tie = false;
    return rawc;
  }
  float wsum = 0.0f, ax = 0.0f, ay = 0.0f, az = 0.0f;
  const uint32_t rc = rawc & 0x00ffffffu;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float4 xi = t.px[(py + i / W) * t.sw + px + i % W];
    const uint32_t ri = t.raw[(py + i / W) * t.sw + px + i % W] & 0x00ffffffu;
    float rh = rcp_approx(L.kappa_scale * agg(i));  // 1 / h_i
    // ||x_C - x_i||_1 or ||x_C - x_i||_2^2: exact integers from the packed
    // bytes (byte-wise |difference|, summed or squared and summed), read as
    // FP32 through the bits of 2^23 + value: the same values the FP32
    // differences give, in two integer instructions and one subtraction
    float u;
    if constexpr (CRIT == kAMNFE) {
      const float d1 = __uint_as_float(__vsadu4(rc, ri) + 0x4B000000u) - 8388608.0f;
      u = d1 * rh;  // ||(x_C - x_i) / h_i||_1
    } else {
      const uint32_t d = __vabsdiffu4(rc, ri);
      const float d2 = __uint_as_float(__dp4a(d, d, 0x4B000000u)) - 8388608.0f;
      u = 0.5f * d2 * (rh * rh);  // 0.5 ||.||_2^2
    }
    float wi = (rh * rh * rh) * expneg<APX, DEG>(L, u);
    wsum += wi;
    ax = fmaf(wi, xi.x, ax);
    ay = fmaf(wi, xi.y, ay);
    az = fmaf(wi, xi.z, az);
  }
  float rw = 1.0f / wsum;
  float yx = ax * rw, yy = ay * rw, yz = az * rw;
  tie = false;
  if (L.stats) {
    auto g = [](float v) { return fabsf(v - floorf(v) - 0.5f); };
    tie = fminf(g(yx), fminf(g(yy), g(yz))) < 1e-3f;
  }
  return pack_rgb(round_u8(yx), round_u8(yy), round_u8(yz), rawc);
}

template <int W, bool REG, int CRIT, int APX, int DEG>
__device__ __forceinline__ uint32_t amnf_pixel(const Launch& L, const TileSmem& t, int px, int py,
                                               int stride, bool& tie) {
  constexpr int N = W * W;
  if constexpr (REG) {
    uint32_t iagg[N];
    l1_aggregates_int<W>(t.raw, t.sw, px, py, iagg);
    float aggr[N];
#pragma unroll
    for (int i = 0; i < N; ++i) aggr[i] = (float)iagg[i];
    return amnf_finish<W, CRIT, APX, DEG>(L, t, px, py, [&](int i) { return aggr[i]; }, tie);
  } else {
    uint32_t* sagg = reinterpret_cast<uint32_t*>(t.agg + threadIdx.x);
    l1_aggregates_int_smem<W>(t.raw, t.sw, px, py, sagg, stride);
    const float* fagg = t.agg + threadIdx.x;
    return amnf_finish<W, CRIT, APX, DEG>(L, t, px, py,
                                          [&](int i) { return fagg[i * stride]; }, tie);
  }
}

// ---------------------------------------------------------------- two windows per thread

// The windows of (px, py) and (px, py + 1) share the w(w - 1) samples of rows
// py + 1 .. py + w - 1.  One thread forms both: the pairs among the shared
// samples once (partial aggregates Cm), then each window's pairs with its own
// extra row (row py for the upper, py + w for the lower window), starting
// from Cm.  Pair terms for the two outputs: m(m - 1)/2 among the m = w(w - 1)
// shared samples plus, per window, w(w - 1)/2 + w m with its extra row: 410
// at w = 5 (205 per output instead of 300), 57 at w = 3 (28.5 instead of 36);
// registers for w <= 5, the rolled form below for w = 7.
// P::pair(a, b, x, y) adds the term of samples a, b to accumulators x and y.
struct PairL1Int {  // AMNF: city-block distance, exact integer sums
  using Acc = uint32_t;
  static __device__ __forceinline__ Acc zero() { return 0u; }
  static __device__ __forceinline__ void pair(uint32_t a, uint32_t b, Acc& x, Acc& y) {
    x = __vsadu4(a, b) + x;
    y = __vsadu4(a, b) + y;
  }
};
struct PairL2 {  // VMF: Euclidean distance, one square root per pair
  using Acc = float;
  static __device__ __forceinline__ Acc zero() { return 0.0f; }
  static __device__ __forceinline__ void pair(uint32_t a, uint32_t b, Acc& x, Acc& y) {
    const float d = TermL2U8{}(a, b);
    x += d;
    y += d;
  }
};

template <int W, class P>
__device__ __forceinline__ void two_window_aggregates(const uint32_t* raw, int sw, int px, int py,
                                                      typename P::Acc (&A)[W * W],
                                                      typename P::Acc (&B)[W * W]) {
  using Acc = typename P::Acc;
  uint32_t X[W + 1][W];  // rows py .. py + w, fourth byte cleared
#pragma unroll
  for (int r = 0; r <= W; ++r)
#pragma unroll
    for (int c = 0; c < W; ++c) X[r][c] = load_sample(raw + (py + r) * sw + px + c);
  Acc Cm[W - 1][W];  // shared rows 1 .. w - 1
#pragma unroll
  for (int r = 0; r < W - 1; ++r)
#pragma unroll
    for (int c = 0; c < W; ++c) Cm[r][c] = P::zero();
#pragma unroll
  for (int r1 = 1; r1 < W; ++r1)
#pragma unroll
    for (int c1 = 0; c1 < W; ++c1) {
#pragma unroll
      for (int c2 = c1 + 1; c2 < W; ++c2)
        P::pair(X[r1][c1], X[r1][c2], Cm[r1 - 1][c1], Cm[r1 - 1][c2]);
#pragma unroll
      for (int r2 = r1 + 1; r2 < W; ++r2)
#pragma unroll
        for (int c2 = 0; c2 < W; ++c2) P::pair(X[r1][c1], X[r2][c2], Cm[r1 - 1][c1], Cm[r2 - 1][c2]);
    }
  // upper window: rows 0 .. w - 1 (A index r * w + c)
#pragma unroll
  for (int r = 1; r < W; ++r)
#pragma unroll
    for (int c = 0; c < W; ++c) A[r * W + c] = Cm[r - 1][c];
  // lower window: rows 1 .. w (B index (r - 1) * w + c)
#pragma unroll
  for (int r = 1; r < W; ++r)
#pragma unroll
    for (int c = 0; c < W; ++c) B[(r - 1) * W + c] = Cm[r - 1][c];
#pragma unroll
  for (int c = 0; c < W; ++c) {
    A[c] = P::zero();
    B[(W - 1) * W + c] = P::zero();
  }
#pragma unroll
  for (int c1 = 0; c1 < W; ++c1) {
#pragma unroll
    for (int c2 = c1 + 1; c2 < W; ++c2) {
      P::pair(X[0][c1], X[0][c2], A[c1], A[c2]);
      P::pair(X[W][c1], X[W][c2], B[(W - 1) * W + c1], B[(W - 1) * W + c2]);
    }
#pragma unroll
    for (int r = 1; r < W; ++r)
#pragma unroll
      for (int c = 0; c < W; ++c) {
        P::pair(X[0][c1], X[r][c], A[c1], A[r * W + c]);
        P::pair(X[W][c1], X[r][c], B[(W - 1) * W + c1], B[(r - 1) * W + c]);
      }
  }
}

// EVMF switch (Sec. 3.3, Eq. equ_evf) of the window of (px, py).  The sample
// loops run row by row; for w <= 5 the n distances r_i stay in registers
// between the sum and the entropy pass, for w = 7 the row loop stays rolled
// and the entropy pass recomputes r_i (one sqrt per sample) instead.
template <int W, int APX, int DEG, bool ALT = false>
__device__ __forceinline__ bool evmf_switch(const Launch& L, const TileSmem& t, int px, int py,
                                            bool& tie) {
  constexpr int N = W * W, C = N / 2;
  constexpr bool KEEP_R = W <= 5;
  constexpr int ROW_UNROLL = KEEP_R ? W : 1;
  // pass 1: the channel sums, exact integers, from the packed pixels: bytes 0
  // and 2 accumulate in the two 16-bit halves of one word, byte 1 in another
  // (n * 255 < 2^16)
  uint32_t s02 = 0, s1 = 0;
#pragma unroll ROW_UNROLL
  for (int a = 0; a < W; ++a) {
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const uint32_t v = t.raw[(py + a) * t.sw + px + i];
      s02 += v & 0x00ff00ffu;
      s1 += (v >> 8) & 0xffu;
    }
  }
  // correctly rounded division: exact whenever the mean is an integer, so a
  // centre equal to the mean gives P_C = 0 exactly (no switch), as in exact
  // arithmetic; a reciprocal multiply would leave a spurious P_C > 0 = beta_C
  const float mx = (float)(s02 & 0xffffu) / (float)N;
  const float my = (float)s1 / (float)N;
  const float mz = (float)(s02 >> 16) / (float)N;
  // pass 2: r_i = ||x_i - xbar||_2 and their sum
  auto dist = [&](int a, int i) {
    float4 xi = t.px[(py + a) * t.sw + px + i];
    float dx = xi.x - mx, dy = xi.y - my, dz = xi.z - mz;
    return sqrt_approx(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  };
  float r[KEEP_R ? N : 1];
  float rsum = 0.0f;
#pragma unroll ROW_UNROLL
  for (int a = 0; a < W; ++a) {
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const float ri = dist(a, i);
      if constexpr (KEEP_R) r[a * W + i] = ri;
      rsum += ri;
    }
  }
  tie = false;
  if (rsum == 0.0f) return false;  // constant window: identity
  const float rs = 1.0f / rsum;
  // pass 3: the entropy sum over P_i = r_i / sum_j r_j
  float esum = 0.0f;
#pragma unroll ROW_UNROLL
  for (int a = 0; a < W; ++a) {
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const float ri = KEEP_R ? r[KEEP_R ? a * W + i : 0] : dist(a, i);
      esum += ent<APX, DEG, ALT>(L, ri * rs);
    }
  }
  if (esum == 0.0f) return false;  // nothing left after the cut-off: identity
  const float4 xc = t.px[(py + C / W) * t.sw + px + C % W];
  const float dx = xc.x - mx, dy = xc.y - my, dz = xc.z - mz;
  const float PC = sqrt_approx(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) * rs;
  const float beta = ent<APX, DEG, ALT>(L, PC) / esum;
  if (L.stats) tie = fabsf(PC - beta) <= 1e-5f * fmaxf(fabsf(PC), fabsf(beta));
  return PC > beta;
}

template <int W, int CRIT, int APX, int DEG, bool REG = uses_reg_path(W, CRIT)>
__device__ __forceinline__ void process_tile(const Launch& L, int tile) {
  constexpr int R = W / 2;
  const int TY = blockDim.x / kTX;
  const TileSmem t = carve(W, REG, TY, blockDim.x);
  const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
  const int x0 = txi * kTX, y0 = tyi * TY;

  stage_tile<CRIT, CRIT != kVMF>(L, t, x0, y0, R);
  __syncthreads();

  const int px = threadIdx.x % kTX, py = threadIdx.x / kTX;
  const int gx = x0 + px, gy = y0 + py;
  const bool valid = gx < L.width && gy < L.height;
  const int stride = blockDim.x;
  float* sagg = t.agg + threadIdx.x;
  const bool want_tie = L.stats != nullptr;
  int ties = 0, switched = 0;

  if constexpr (CRIT == kVMF || CRIT == kBVDF) {
    Selection s;
    if constexpr (CRIT == kVMF) {
      s = window_select<W, REG>(t.raw, t.sw, px, py, TermL2U8{}, sagg, stride, want_tie);
    } else if constexpr (APX == kExact) {
      s = window_select<W, REG>(t.px, t.sw, px, py, TermAngleExact(L.c.a), sagg, stride, want_tie);
    } else {
      s = window_select<W, REG>(t.px, t.sw, px, py, TermAngleApprox<DEG>(L.c.a, L.c.b), sagg, stride,
                           want_tie);
    }
    if (valid) {
      store_px(L, gx, gy, t.raw[(py + s.best / W) * t.sw + px + s.best % W]);
      ties = s.near_tie;
    }
  } else if constexpr (CRIT == kAMNFE || CRIT == kAMNFG) {
    bool tie = false;
    uint32_t v = amnf_pixel<W, REG, CRIT, APX, DEG>(L, t, px, py, stride, tie);
    if (valid) {
      store_px(L, gx, gy, v);
      ties = tie;
    }
  } else {  // kEVMF / kEVBDF: switch, then the selection on the compacted list
    __shared__ int s_count;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    bool tie = false;
    bool sw = valid && evmf_switch<W, APX, DEG, CRIT == kEVBDF>(L, t, px, py, tie);
    if (valid && !sw) store_px(L, gx, gy, t.raw[(py + R) * t.sw + px + R]);
    if (sw) t.list[atomicAdd(&s_count, 1)] = threadIdx.x;
    ties = valid && tie;
    switched = sw;
    __syncthreads();
    const int count = s_count;
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
      const int id = t.list[k];
      const int qx = id % kTX, qy = id / kTX;
      Selection s;
      if constexpr (CRIT == kEVMF) {
        s = window_select<W, REG>(t.raw, t.sw, qx, qy, TermL2U8{}, sagg, stride, want_tie);
      } else if constexpr (APX == kExact) {  // EVBDF: the angle of Sec. 3.1
        s = window_select<W, REG>(t.px, t.sw, qx, qy, TermAngleExact(L.c.a), sagg, stride, want_tie);
      } else {
        s = window_select<W, REG>(t.px, t.sw, qx, qy, TermAngleApprox<DEG>(L.c.a, L.c.b), sagg,
                                  stride, want_tie);
      }
      store_px(L, x0 + qx, y0 + qy, t.raw[(qy + s.best / W) * t.sw + qx + s.best % W]);
      ties += s.near_tie;
    }
  }
  block_stats(L, valid ? 1 : 0, ties, switched);
}

// The same two windows with the row loops rolled and the aggregates in
// shared-memory slots sA[i * stride], sB[i * stride] (w = 7, where n = 49
// register aggregates per window would not fit): the shared rows' pairs go to
// the upper window's slots, which are then copied to the lower window's, and
// each window adds the pairs of its own extra row.  Pair terms per output at
// w = 7: 745.5 instead of 1176.
template <int W, class P>
__device__ __forceinline__ void two_window_extra_row(const uint32_t* raw, int sw, int px, int py,
                                                     int extra, int row_lo,
                                                     typename P::Acc* slots, int stride) {
  // `extra`: the extra row's offset from py (0 or w); `row_lo`: the slot row
  // of tile row py + 1 (1 for the upper window, 0 for the lower); the extra
  // row's own slots are row 0 (upper) or w - 1 (lower)
  using Acc = typename P::Acc;
  const int own = extra == 0 ? 0 : W - 1;
  uint32_t E[W];
  Acc re[W];
#pragma unroll
  for (int c = 0; c < W; ++c) {
    E[c] = load_sample(raw + (py + extra) * sw + px + c);
    re[c] = P::zero();
  }
#pragma unroll
  for (int c1 = 0; c1 < W; ++c1)
#pragma unroll
    for (int c2 = c1 + 1; c2 < W; ++c2) P::pair(E[c1], E[c2], re[c1], re[c2]);
#pragma unroll 1
  for (int r = 1; r < W; ++r) {
    uint32_t Y[W];
    Acc ry[W];
#pragma unroll
    for (int c = 0; c < W; ++c) {
      Y[c] = load_sample(raw + (py + r) * sw + px + c);
      ry[c] = P::zero();
    }
#pragma unroll
    for (int c1 = 0; c1 < W; ++c1)
#pragma unroll
      for (int c2 = 0; c2 < W; ++c2) P::pair(E[c1], Y[c2], re[c1], ry[c2]);
    Acc* row = slots + (row_lo + r - 1) * W * stride;
#pragma unroll
    for (int c = 0; c < W; ++c) row[c * stride] += ry[c];
  }
#pragma unroll
  for (int c = 0; c < W; ++c) slots[(own * W + c) * stride] = re[c];
}

template <int W, class P>
__device__ __forceinline__ void two_window_aggregates_smem(const uint32_t* raw, int sw, int px,
                                                           int py, typename P::Acc* sA,
                                                           typename P::Acc* sB, int stride) {
  using Acc = typename P::Acc;
#pragma unroll
  for (int i = 0; i < W * W; ++i) sA[i * stride] = P::zero();
  // pairs of the shared rows py + 1 .. py + w - 1 into the upper window's slots
#pragma unroll 1
  for (int a = 1; a < W; ++a) {
    uint32_t X[W];
    Acc ra[W];
#pragma unroll
    for (int c = 0; c < W; ++c) {
      X[c] = load_sample(raw + (py + a) * sw + px + c);
      ra[c] = P::zero();
    }
#pragma unroll
    for (int c1 = 0; c1 < W; ++c1)
#pragma unroll
      for (int c2 = c1 + 1; c2 < W; ++c2) P::pair(X[c1], X[c2], ra[c1], ra[c2]);
#pragma unroll 1
    for (int b = a + 1; b < W; ++b) {
      uint32_t Y[W];
      Acc rb[W];
#pragma unroll
      for (int c = 0; c < W; ++c) {
        Y[c] = load_sample(raw + (py + b) * sw + px + c);
        rb[c] = P::zero();
      }
#pragma unroll
      for (int c1 = 0; c1 < W; ++c1)
#pragma unroll
        for (int c2 = 0; c2 < W; ++c2) P::pair(X[c1], Y[c2], ra[c1], rb[c2]);
#pragma unroll
      for (int c = 0; c < W; ++c) sA[(b * W + c) * stride] += rb[c];
    }
#pragma unroll
    for (int c = 0; c < W; ++c) sA[(a * W + c) * stride] += ra[c];
  }
  // the lower window starts from the same shared-row sums
#pragma unroll 1
  for (int r = 1; r < W; ++r)
#pragma unroll
    for (int c = 0; c < W; ++c) sB[((r - 1) * W + c) * stride] = sA[(r * W + c) * stride];
  two_window_extra_row<W, P>(raw, sw, px, py, 0, 1, sA, stride);  // row py: upper window
  two_window_extra_row<W, P>(raw, sw, px, py, W, 0, sB, stride);  // row py + w: lower window
}

// Per-window VMF / AMNF with two outputs per thread (w <= 5): a CTA of
// 32 x T threads covers a 32 x 2T tile, thread (px, r) the windows of rows 2r
// and 2r + 1, formed together by two_window_aggregates.
template <int W, int CRIT, int APX, int DEG>
__device__ __forceinline__ void process_tile2(const Launch& L, int tile) {
  constexpr int R = W / 2, N = W * W;
  constexpr bool REG = uses_reg_path(W, CRIT);
  const int TY = 2 * (blockDim.x / kTX);
  // rolled form: 2 x n slots per thread (upper and lower window)
  const TileSmem t = carve(W, REG, TY, REG ? blockDim.x : 2 * blockDim.x);
  const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
  const int x0 = txi * kTX, y0 = tyi * TY;
  stage_tile<CRIT, CRIT != kVMF>(L, t, x0, y0, R);
  __syncthreads();
  const int px = threadIdx.x % kTX, py = 2 * (threadIdx.x / kTX);
  const int gx = x0 + px, gy = y0 + py;
  const bool va = gx < L.width && gy < L.height;
  const bool vb = gx < L.width && gy + 1 < L.height;
  int ties = 0;
  const int T = blockDim.x;
  if constexpr (CRIT == kVMF) {
    const bool want_tie = L.stats != nullptr;
    Selection sa, sb;
    if constexpr (REG) {
      float A[N], B[N];
      two_window_aggregates<W, PairL2>(t.raw, t.sw, px, py, A, B);
      sa = select_min<W, true>(A, nullptr, 0, t.raw, t.sw, px, py, want_tie);
      sb = select_min<W, true>(B, nullptr, 0, t.raw, t.sw, px, py + 1, want_tie);
    } else {
      float* sA = t.agg + threadIdx.x;
      float* sB = sA + N * T;
      two_window_aggregates_smem<W, PairL2>(t.raw, t.sw, px, py, sA, sB, T);
      sa = select_min<W, false>(nullptr, sA, T, t.raw, t.sw, px, py, want_tie);
      sb = select_min<W, false>(nullptr, sB, T, t.raw, t.sw, px, py + 1, want_tie);
    }
    if (va) {
      store_px(L, gx, gy, t.raw[(py + sa.best / W) * t.sw + px + sa.best % W]);
      ties += sa.near_tie;
    }
    if (vb) {
      store_px(L, gx, gy + 1, t.raw[(py + 1 + sb.best / W) * t.sw + px + sb.best % W]);
      ties += sb.near_tie;
    }
  } else {
    bool ta = false, tb = false;
    uint32_t oa, ob;
    if constexpr (REG) {
      uint32_t A[N], B[N];
      two_window_aggregates<W, PairL1Int>(t.raw, t.sw, px, py, A, B);
      oa = amnf_finish<W, CRIT, APX, DEG>(L, t, px, py, [&](int i) { return (float)A[i]; }, ta);
      ob = amnf_finish<W, CRIT, APX, DEG>(L, t, px, py + 1, [&](int i) { return (float)B[i]; },
                                          tb);
    } else {  // integer sums in the float slots' storage
      uint32_t* sA = reinterpret_cast<uint32_t*>(t.agg + threadIdx.x);
      uint32_t* sB = sA + N * T;
      two_window_aggregates_smem<W, PairL1Int>(t.raw, t.sw, px, py, sA, sB, T);
      oa = amnf_finish<W, CRIT, APX, DEG>(L, t, px, py, [&](int i) { return (float)sA[i * T]; },
                                          ta);
      ob = amnf_finish<W, CRIT, APX, DEG>(L, t, px, py + 1,
                                          [&](int i) { return (float)sB[i * T]; }, tb);
    }
    if (va) {
      store_px(L, gx, gy, oa);
      ties += ta;
    }
    if (vb) {
      store_px(L, gx, gy + 1, ob);
      ties += tb;
    }
  }
  block_stats(L, (int)va + (int)vb, ties, 0);
}

template <int W, int CRIT, int APX, int DEG>
__global__ void __launch_bounds__(256) filter2_kernel(const __grid_constant__ Launch L) {
  pdl_begin();
  process_tile2<W, CRIT, APX, DEG>(L, blockIdx.x);
}

// One CTA per tile of one image.
template <int W, int CRIT, int APX, int DEG>
__global__ void __launch_bounds__(256) filter_kernel(const __grid_constant__ Launch L) {
  pdl_begin();
  process_tile<W, CRIT, APX, DEG>(L, blockIdx.x);
}

}  // namespace vf
