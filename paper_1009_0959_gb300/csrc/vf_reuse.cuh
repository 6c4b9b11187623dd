// vf_reuse.cuh -- window kernels that compute every pairwise term once per
// tile instead of once per window (cross-window reuse).
//
// A pair of pixels (p, q) with |p - q| <= w - 1 (per axis) belongs to every
// window that contains both, up to w^2 of them; the per-window kernel
// computes it in each.  Here a CTA of 32 x RTY outputs (RTY = 8, or taller
// tiles with one thread per region pixel) stages its
// (32 + w - 1) x (RTY + w - 1) region once, then
//   1. term table: for every region pixel p and each of the 2w(w-1) offsets
//      delta of the forward half-plane (dy > 0, or dy = 0 and dx > 0) with
//      p + delta in the region, T[delta][p] = term(x_p, x_{p+delta});
//   2. aggregates: every region pixel p forms, for each window c containing p,
//      agg(c, p) = sum_{q in W(c)} term(p, q) as separable box sums of its
//      distance field D_p(delta) (T[delta][p] or T[-delta][p + delta], 0 at
//      delta = 0) over the (2w-1)^2 offsets: row sums of width w, then column
//      sums of height w.  Only additions at w = 3 and 5 (no differences of
//      prefix sums, so no cancellation); the 7 x 7 register form slides its
//      width-7 row sums (one addition and one subtraction of non-negative
//      terms per step);
//   3. every output thread reads the n aggregates of its window and selects
//      (argmin, lowest index) or weights (AMNF), as the per-window kernel.
// Work per output pixel: 2w(w-1) terms x (region / tile) instead of
// n(n-1)/2, plus O(w^3) additions.  The aggregates are the same sums in
// another order (FP32, relative differences of a few 1e-7).
#pragma once

#include <algorithm>
#include <type_traits>

#include "vf_kernels.cuh"

namespace vf {

constexpr int kRTX = 32, kRTY = 8;  // outputs per reuse tile

template <int W, int RTY = kRTY, int NT = kRTX * RTY>
struct ReuseGeom {
  static constexpr int R = W / 2;
  static constexpr int RX = kRTX + W - 1;     // region columns
  static constexpr int RY = RTY + W - 1;      // region rows
  static constexpr int NR = RX * RY;          // region pixels
  static constexpr int N = W * W;             // window samples
  static constexpr int M = W - 1;             // largest offset per axis
  static constexpr int ND = M * (2 * M + 1) + M;  // forward half-plane offsets = 2w(w-1)
  static constexpr int THREADS = NT;         // threads of the CTA
  static constexpr int OUT = kRTX * RTY;      // outputs of the tile
};

// Calls f(std::integral_constant<int, k>{}) for k = A .. B in order.
template <int A, int B, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (A <= B) {
    f(std::integral_constant<int, A>{});
    static_for<A + 1, B>(f);
  }
}

__host__ __device__ constexpr size_t reuse_smem_bytes(int w, int rty = kRTY) {
  size_t rx = kRTX + w - 1, ry = rty + w - 1, nr = rx * ry, m = w - 1;
  size_t nd = m * (2 * m + 1) + m;
  return nr * 20 + nd * nr * 4 + (size_t)w * w * kRTX * rty * 4;
}

// Threads of a reuse CTA: one per output at 8 rows; for taller tiles one per
// region pixel (rounded up to whole warps), so that the term items and the
// box sums of phase 2 split into whole rounds
constexpr int reuse_threads(int w, int rty) {
  return rty == kRTY ? kRTX * rty : ((kRTX + w - 1) * (rty + w - 1) + 31) / 32 * 32;
}

// index of forward offset (dy, dx): dy = 0 -> dx - 1; dy > 0 -> M + (dy-1)(2M+1) + dx + M
template <int W>
__host__ __device__ constexpr int fwd_index(int dy, int dx) {
  return dy == 0 ? dx - 1 : (W - 1) + (dy - 1) * (2 * (W - 1) + 1) + dx + (W - 1);
}

// Phase 3 of the reuse kernels: each output thread reads the n aggregates
// of its window from the slots A[i * OUT + output] and selects (argmin,
// lowest index) or weights (AMNF) exactly as the per-window kernel does.
// Threads beyond the tile's outputs only join the counters' reduction.
template <int W, int CRIT, int APX, int DEG, int RTY = kRTY, int NT = kRTX * RTY>
__device__ __forceinline__ void reuse_finish(const Launch& L, const float4* px,
                                             const uint32_t* raw, const float* A, int x0,
                                             int y0) {
  using G = ReuseGeom<W, RTY, NT>;
  constexpr int R = G::R, RX = G::RX, N = G::N;
  const int ox = threadIdx.x % kRTX, oy = threadIdx.x / kRTX;
  const int gx = x0 + ox, gy = y0 + oy;
  const bool mine = (int)threadIdx.x < G::OUT;
  const bool valid = mine && gx < L.width && gy < L.height;
  // gated form: only flagged outputs are filtered, the others keep the centre
  const bool on = valid && (L.flags == nullptr || L.flags[(long long)gy * L.flag_pitch + gx] != 0);
  const float* sagg = A + threadIdx.x;
  int ties = 0, switched = 0;
  if (!mine) {
  } else if constexpr (CRIT == kAMNFE || CRIT == kAMNFG) {
    const float4 xc = px[(oy + R) * RX + ox + R];
    const uint32_t rawc = raw[(oy + R) * RX + ox + R];
    uint32_t v = rawc;
    if (sagg[(N / 2) * G::OUT] != 0.0f) {  // not a constant window
      float wsum = 0.0f, ax = 0.0f, ay = 0.0f, az = 0.0f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float4 xi = px[(oy + i / W) * RX + ox + i % W];
        const float rh = rcp_approx(L.kappa_scale * sagg[i * G::OUT]);
        const float dx = xc.x - xi.x, dy = xc.y - xi.y, dz = xc.z - xi.z;
        float u;
        if constexpr (CRIT == kAMNFE) {
          u = (fabsf(dx) + fabsf(dy) + fabsf(dz)) * rh;
        } else {
          u = 0.5f * fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * (rh * rh);
        }
        const float wi = (rh * rh * rh) * expneg<APX, DEG>(L, u);
        wsum += wi;
        ax = fmaf(wi, xi.x, ax);
        ay = fmaf(wi, xi.y, ay);
        az = fmaf(wi, xi.z, az);
      }
      const float rw = 1.0f / wsum;
      const float yx = ax * rw, yy = ay * rw, yz = az * rw;
      if (L.stats) {
        auto g = [](float q) { return fabsf(q - floorf(q) - 0.5f); };
        ties = fminf(g(yx), fminf(g(yy), g(yz))) < 1e-3f;
      }
      v = pack_rgb(round_u8(yx), round_u8(yy), round_u8(yz), rawc);
    }
    if (valid) store_px(L, gx, gy, on ? v : rawc);
    ties = on ? ties : 0;
  } else if constexpr (CRIT == kEVMF || CRIT == kEVBDF) {
    // the EVMF (Eq. equ_evf) and the generalised EVF: the entropy switch on
    // this output's window (the staged region is laid out as a per-window
    // tile of pitch RX), the vector median (EVMF: Euclidean aggregates) or
    // BVDF's selection (EVBDF: angle aggregates) when it fires, the centre
    // otherwise
    TileSmem ts;
    ts.px = const_cast<float4*>(px);
    ts.raw = const_cast<uint32_t*>(raw);
    ts.sw = RX;
    ts.sh = G::RY;
    bool tie = false;
    const bool sw = valid && evmf_switch<W, APX, DEG, CRIT == kEVBDF>(L, ts, ox, oy, tie);
    uint32_t v = raw[(oy + R) * RX + ox + R];
    if (sw) {
      const Selection s =
          select_min<W, false>(nullptr, sagg, G::OUT, px, RX, ox, oy, L.stats != nullptr);
      v = raw[(oy + s.best / W) * RX + ox + s.best % W];
      tie = tie || s.near_tie;
    }
    if (valid) store_px(L, gx, gy, v);
    ties = tie;
    switched = sw;
  } else {
    const Selection s =
        select_min<W, false>(nullptr, sagg, G::OUT, px, RX, ox, oy, L.stats != nullptr);
    const int pick = on ? s.best : N / 2;
    if (valid) store_px(L, gx, gy, raw[(oy + pick / W) * RX + ox + pick % W]);
    ties = on && s.near_tie;
  }
  // gated form: the third counter counts the filtered pixels
  if (L.flags != nullptr) switched = on;
  block_stats(L, valid ? 1 : 0, valid ? ties : 0, switched);
}

// Gated form: a tile none of whose outputs is flagged is copied without
// staging or pair terms.  Called by every thread (the test is a barrier);
// true when the tile was copied.
template <int RTY, int NT>
__device__ __forceinline__ bool reuse_gated_skip(const Launch& L, int tile) {
  constexpr int OUT = kRTX * RTY;
  const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
  const int x0 = txi * kRTX, y0 = tyi * RTY;
  int any = 0;
  for (int o = threadIdx.x; o < OUT; o += NT) {
    const int gx = x0 + o % kRTX, gy = y0 + o / kRTX;
    if (gx < L.width && gy < L.height) any |= L.flags[(long long)gy * L.flag_pitch + gx] != 0;
  }
  if (__syncthreads_or(any)) return false;
  int pixels = 0;
  for (int o = threadIdx.x; o < OUT; o += NT) {
    const int gx = x0 + o % kRTX, gy = y0 + o / kRTX;
    if (gx < L.width && gy < L.height) {
      store_px(L, gx, gy, load_px(L, gx, gy));
      ++pixels;
    }
  }
  block_stats(L, pixels, 0, 0);
  return true;
}

// The same, not inlined: for the 7 x 7 tiles, whose 49 register window sums
// leave no room for the test's values (inlined, it made the main loop spill).
template <int RTY, int NT>
__device__ __noinline__ bool reuse_gated_skip_call(const Launch& L, int tile) {
  return reuse_gated_skip<RTY, NT>(L, tile);
}

// The w sums of w consecutive values of v[0 .. 2w-2]: out[e] = v[e] + ... +
// v[e + w - 1].  Neighbouring sums share their overlap (w = 5: 12 additions
// instead of 20); additions only.
template <int W>
__device__ __forceinline__ void box_sums(const float (&v)[2 * W - 1], float (&out)[W]) {
  if constexpr (W == 5) {
    const float m1 = (v[1] + v[2]) + (v[3] + v[4]);
    out[0] = v[0] + m1;
    out[1] = m1 + v[5];
    const float q = (v[4] + v[5]) + v[6];
    const float m3 = v[3] + q;
    out[2] = v[2] + m3;
    out[3] = m3 + v[7];
    out[4] = q + (v[7] + v[8]);
  } else if constexpr (W == 3) {
    const float m = v[1] + v[2];
    out[0] = v[0] + m;
    out[1] = m + v[3];
    out[2] = (v[2] + v[3]) + v[4];
  } else {
#pragma unroll
    for (int e = 0; e < W; ++e) {
      float t = 0.0f;
#pragma unroll
      for (int k = 0; k < W; ++k) t += v[e + k];
      out[e] = t;
    }
  }
}

// Phases 1-3 of a tile whose region is staged (px, raw) and visible to the
// whole CTA.
template <int W, int CRIT, int APX, int DEG, int RTY = kRTY, int NT = kRTX * RTY>
__device__ __forceinline__ void reuse_tile_body(const Launch& L, int tile) {
  using G = ReuseGeom<W, RTY, NT>;
  constexpr int R = G::R, RX = G::RX, RY = G::RY, NR = G::NR, M = G::M, ND = G::ND;
  extern __shared__ __align__(16) unsigned char smem[];
  float4* px = reinterpret_cast<float4*>(smem);
  uint32_t* raw = reinterpret_cast<uint32_t*>(smem + NR * 16);
  float* T = reinterpret_cast<float*>(smem + NR * 20);   // [ND][NR]
  float* A = T + ND * NR;                                  // [N][OUT]
  const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
  const int x0 = txi * kRTX, y0 = tyi * RTY;

  // 1. term table.  Entries whose partner p + delta lies outside the region
  //    (past its last row, or across its left or right edge, where the flat
  //    index wraps to another row) belong to no window of the tile: phase 2
  //    reads them only into sums for windows that are discarded (below), so
  //    their values do not matter.  Work items are (offset column dx, region
  //    pixel p), w - 1 or w terms each (dy = 0 only for dx > 0): (2w - 1) x
  //    region items of nearly equal cost, so the last round leaves few
  //    threads idle.
  auto row_terms = [&](const auto& term, const auto* src) {
    if constexpr (NT >= NR) {
      // one thread per region pixel: every offset is a compile-time constant
      // and the pixel's own sample is loaded once; no bound test (a partner
      // past the region's end reads the next shared array)
      const int p = threadIdx.x;
      if (p >= NR) return;
      const auto xp = load_sample(src + p);
      auto one = [&](auto DX) {
        constexpr int dx = decltype(DX)::value;
#pragma unroll
        for (int dy = 0; dy <= M; ++dy) {
          if (dy == 0 && dx <= 0) continue;
          T[fwd_index<W>(dy, dx) * NR + p] = term(xp, load_sample(src + p + dy * RX + dx));
        }
      };
      static_for<-M, M>(one);
    } else {
      for (int item = threadIdx.x; item < (2 * M + 1) * NR; item += G::THREADS) {
        const int dxi = item / NR, p = item - dxi * NR;
        const int dx = dxi - M;
        const int r = p / RX, c = p - r * RX;
        const bool col_in = c + dx >= 0 && c + dx < RX;
        const auto xp = load_sample(src + p);
#pragma unroll
        for (int dy = 0; dy <= M; ++dy) {
          if (dy == 0 && dx <= 0) continue;
          float v = 0.0f;
          if (col_in && r + dy < RY) v = term(xp, load_sample(src + p + dy * RX + dx));
          T[fwd_index<W>(dy, dx) * NR + p] = v;
        }
      }
    }
  };
  if constexpr (CRIT == kVMF || CRIT == kEVMF) {
    row_terms(TermL2U8{}, raw);  // packed bytes: exact squared distances
  } else if constexpr (CRIT == kAMNFE || CRIT == kAMNFG) {
    row_terms(TermL1{}, px);
  } else if constexpr (APX == kExact) {
    row_terms(TermAngleExact(L.c.a), px);
  } else {
    row_terms(TermAngleApprox<DEG>(L.c.a, L.c.b), px);
  }
  __syncthreads();

  // 2. box sums of each region pixel's distance field, scattered to the
  //    windows of this tile that contain it: width-w sums along each of the
  //    2w - 1 field rows, then height-w sums down the columns, both sharing
  //    their common partial sums (additions only).  A window that is kept
  //    (its output inside the tile) holds only partners inside the region,
  //    and each of its sums is an exact expression over its own field
  //    entries (the shared partial sums are sums of subsets of both), so the
  //    entries of partners outside the region -- forward entries never
  //    zeroed, mirrored reads that wrap across a region edge or start up to
  //    (w - 1)(RX + 1) floats before a table row (in the packed pixels'
  //    array) -- reach only discarded windows, and need no bound test.
  for (int p = threadIdx.x; p < NR; p += G::THREADS) {
    const int r = p / RX, c = p - r * RX;
    float h[2 * M + 1][W];  // h[dy + M][ex + R]: field row dy summed over dx in ex +- R
#pragma unroll
    for (int dy = -M; dy <= M; ++dy) {
      float d[2 * M + 1];
#pragma unroll
      for (int dx = -M; dx <= M; ++dx) {
        if (dy > 0 || (dy == 0 && dx > 0)) {
          d[dx + M] = T[fwd_index<W>(dy, dx) * NR + p];
        } else if (dy == 0 && dx == 0) {
          d[dx + M] = 0.0f;
        } else {
          d[dx + M] = T[fwd_index<W>(-dy, -dx) * NR + p + dy * RX + dx];
        }
      }
      box_sums<W>(d, h[dy + M]);
    }
    // window centred at region (r + ey, c + ex) = output (r + ey - R, c + ex - R)
#pragma unroll
    for (int ex = -R; ex <= R; ++ex) {
      float col[2 * M + 1], v[W];
#pragma unroll
      for (int k = 0; k <= 2 * M; ++k) col[k] = h[k][ex + R];
      box_sums<W>(col, v);
      const int ox = c + ex - R;
#pragma unroll
      for (int ey = -R; ey <= R; ++ey) {
        const int oy = r + ey - R;
        if (oy >= 0 && oy < RTY && ox >= 0 && ox < kRTX) {
          const int j = (R - ey) * W + (R - ex);  // p's index in that window
          A[j * G::OUT + oy * kRTX + ox] = v[ey + R];
        }
      }
    }
  }
  __syncthreads();

  // 3. selection / weighting per output
  reuse_finish<W, CRIT, APX, DEG, RTY, NT>(L, px, raw, A, x0, y0);
}

template <int W, int CRIT, int APX, int DEG, int RTY = kRTY, int NT = kRTX * RTY>
__device__ __forceinline__ void reuse_tile(const Launch& L, int tile) {
  using G = ReuseGeom<W, RTY, NT>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
  TileSmem t;
  t.px = reinterpret_cast<float4*>(smem);
  t.raw = reinterpret_cast<uint32_t*>(smem + G::NR * 16);
  t.sw = G::RX;
  t.sh = G::RY;
  stage_tile<CRIT>(L, t, txi * kRTX, tyi * RTY, G::R);
  __syncthreads();
  reuse_tile_body<W, CRIT, APX, DEG, RTY, NT>(L, tile);
}

// Chunked form for large windows, where the whole term table would not fit in
// shared memory next to a useful occupancy (w = 7: 84 x 532 floats).  The
// table is built one forward offset row dy = k at a time (2w - 1 entries per
// pixel); after each row every region pixel adds the box-sum contributions of
// its distance field's rows +k and -k (the latter from the mirrored entries
// T_k[-dx][p + (-k, dx)]) directly to the per-window slots A, which therefore
// accumulate in shared memory instead of registers.  Same sums, another
// order.
inline size_t reuse_chunked_smem_bytes(int w) {
  size_t rx = kRTX + w - 1, ry = kRTY + w - 1, nr = rx * ry;
  return nr * 20 + (size_t)(2 * w - 1) * nr * 4 + (size_t)w * w * kRTX * kRTY * 4;
}

template <int W, int CRIT, int APX, int DEG>
__device__ __forceinline__ void reuse_chunked_tile(const Launch& L, int tile) {
  using G = ReuseGeom<W>;
  constexpr int R = G::R, RX = G::RX, RY = G::RY, NR = G::NR, N = G::N, M = G::M;
  constexpr int ROW = 2 * M + 1;  // entries of one offset row
  extern __shared__ __align__(16) unsigned char smem[];
  float4* px = reinterpret_cast<float4*>(smem);
  uint32_t* raw = reinterpret_cast<uint32_t*>(smem + NR * 16);
  float* T = reinterpret_cast<float*>(smem + NR * 20);  // [ROW][NR]: T[dx + M][p]
  float* A = T + ROW * NR;                                // [N][THREADS]
  const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
  const int x0 = txi * kRTX, y0 = tyi * kRTY;

  TileSmem t;
  t.px = px;
  t.raw = raw;
  t.sw = RX;
  t.sh = RY;
  stage_tile<CRIT>(L, t, x0, y0, R);
  for (int k = threadIdx.x; k < N * G::THREADS; k += G::THREADS) A[k] = 0.0f;
  __syncthreads();

  // adds the box sums of one field row dy (values d[dx + M]) of region pixel
  // (r, c) to the slots of the tile's windows that contain the pixel
  auto add_row = [&](int r, int c, int dy, const float (&d)[ROW]) {
    float h[W];
#pragma unroll
    for (int ex = -R; ex <= R; ++ex) {
      float s = 0.0f;
#pragma unroll
      for (int q = ex - R; q <= ex + R; ++q) s += d[q + M];
      h[ex + R] = s;
    }
#pragma unroll
    for (int ey = -R; ey <= R; ++ey) {
      if (dy < ey - R || dy > ey + R) continue;
      const int oy = r + ey - R;
      if (oy < 0 || oy >= kRTY) continue;
#pragma unroll
      for (int ex = -R; ex <= R; ++ex) {
        const int ox = c + ex - R;
        if (ox >= 0 && ox < kRTX) {
          const int j = (R - ey) * W + (R - ex);
          A[j * G::THREADS + oy * kRTX + ox] += h[ex + R];
        }
      }
    }
  };

  for (int k = 0; k <= M; ++k) {
    // term row k: T[dx + M][p] = term(x_p, x_{p + (k, dx)})
    auto row_terms = [&](const auto& term) {
      for (int p = threadIdx.x; p < NR; p += G::THREADS) {
        const int r = p / RX, c = p - r * RX;
        if (r + k >= RY) continue;
        const float4 xp = px[p];
#pragma unroll
        for (int dx = -M; dx <= M; ++dx) {
          if (k == 0 && dx <= 0) continue;
          if (c + dx >= 0 && c + dx < RX) T[(dx + M) * NR + p] = term(xp, px[p + k * RX + dx]);
        }
      }
    };
    if constexpr (CRIT == kVMF || CRIT == kEVMF) {
      row_terms(TermL2{});
    } else if constexpr (CRIT == kAMNFE || CRIT == kAMNFG) {
      row_terms(TermL1{});
    } else if constexpr (APX == kExact) {
      row_terms(TermAngleExact(L.c.a));
    } else {
      row_terms(TermAngleApprox<DEG>(L.c.a, L.c.b));
    }
    __syncthreads();
    // field rows +k and -k of every region pixel
    for (int p = threadIdx.x; p < NR; p += G::THREADS) {
      const int r = p / RX, c = p - r * RX;
      float d[ROW];
      if (k == 0) {
#pragma unroll
        for (int dx = -M; dx <= M; ++dx) {
          const int cq = c + dx;
          float v = 0.0f;
          if (cq >= 0 && cq < RX) {
            if (dx > 0) v = T[(dx + M) * NR + p];
            else if (dx < 0) v = T[(-dx + M) * NR + p + dx];
          }
          d[dx + M] = v;
        }
        add_row(r, c, 0, d);
      } else {
#pragma unroll
        for (int dx = -M; dx <= M; ++dx) {
          const int cq = c + dx;
          d[dx + M] = (r + k < RY && cq >= 0 && cq < RX) ? T[(dx + M) * NR + p] : 0.0f;
        }
        add_row(r, c, k, d);
#pragma unroll
        for (int dx = -M; dx <= M; ++dx) {
          const int rq = r - k, cq = c + dx;
          d[dx + M] = (rq >= 0 && cq >= 0 && cq < RX) ? T[(-dx + M) * NR + rq * RX + cq] : 0.0f;
        }
        add_row(r, c, -k, d);
      }
    }
    __syncthreads();
  }
  reuse_finish<W, CRIT, APX, DEG>(L, px, raw, A, x0, y0);
}

// The chunked form with one thread per region pixel (NT >= NR): every thread
// keeps the w^2 box sums of its own distance field in registers across the
// offset rows and writes them to the window slots once at the end, instead
// of adding each field row's contributions to the slots in shared memory
// (w^2 read-modify-writes per field row).  Same sums, another order.
__host__ __device__ constexpr size_t reuse_chunked_reg_smem_bytes(int w, int rty) {
  size_t rx = kRTX + w - 1, ry = rty + w - 1, nr = rx * ry;
  return nr * 20 + (size_t)(2 * w - 1) * nr * 4 + (size_t)w * w * kRTX * rty * 4;
}

// The tile's phases once its region is staged (px, raw) and visible.
template <int W, int CRIT, int APX, int DEG, int RTY, int NT>
__device__ __forceinline__ void reuse_chunked_reg_tile_body(const Launch& L, int tile) {
  using G = ReuseGeom<W, RTY, NT>;
  constexpr int R = G::R, RX = G::RX, RY = G::RY, NR = G::NR, M = G::M;
  constexpr int ROW = 2 * M + 1;  // entries of one offset row
  static_assert(NT >= NR, "one thread per region pixel");
  extern __shared__ __align__(16) unsigned char smem[];
  float4* px = reinterpret_cast<float4*>(smem);
  uint32_t* raw = reinterpret_cast<uint32_t*>(smem + NR * 16);
  float* T = reinterpret_cast<float*>(smem + NR * 20);  // [ROW][NR]: T[dx + M][p]
  float* A = T + ROW * NR;                                // [N][OUT]
  const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
  const int x0 = txi * kRTX, y0 = tyi * RTY;

  const int p = threadIdx.x;
  const bool mine = p < NR;
  const int r = p / RX, c = p - r * RX;
  float agg[W][W];  // [ey + R][ex + R]: window centred at region (r + ey, c + ex)
#pragma unroll
  for (int i = 0; i < W; ++i)
#pragma unroll
    for (int j = 0; j < W; ++j) agg[i][j] = 0.0f;
  // adds field row dy (values d[dx + M]) to the windows whose rows hold it
  auto add_row = [&](int dy, const float (&d)[ROW]) {
    float h[W];  // h[ex + R] = d[ex - R + M] + ... + d[ex + R + M], a sliding sum
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < W; ++q) s += d[q];
    h[0] = s;
#pragma unroll
    for (int ex = -R + 1; ex <= R; ++ex) {
      s += d[ex + R + M] - d[ex - R - 1 + M];
      h[ex + R] = s;
    }
#pragma unroll
    for (int ey = -R; ey <= R; ++ey) {
      if (dy < ey - R || dy > ey + R) continue;
#pragma unroll
      for (int ex = -R; ex <= R; ++ex) agg[ey + R][ex + R] += h[ex + R];
    }
  };

#pragma unroll 1
  for (int k = 0; k <= M; ++k) {
    // term row k: T[dx + M][p] = term(x_p, x_{p + (k, dx)}), 0 outside the region
    auto row_terms = [&](const auto& term, const auto* src) {
      if (!mine) return;
      const bool row_in = r + k < RY;
      const auto xp = load_sample(src + p);
#pragma unroll
      for (int dx = -M; dx <= M; ++dx) {
        if (k == 0 && dx <= 0) continue;
        float v = 0.0f;
        if (row_in && c + dx >= 0 && c + dx < RX) v = term(xp, load_sample(src + p + k * RX + dx));
        T[(dx + M) * NR + p] = v;
      }
    };
    if constexpr (CRIT == kVMF || CRIT == kEVMF) {
      row_terms(TermL2U8{}, raw);
    } else if constexpr (CRIT == kAMNFE || CRIT == kAMNFG) {
      row_terms(TermL1{}, px);
    } else if constexpr (APX == kExact) {
      row_terms(TermAngleExact(L.c.a), px);
    } else {
      row_terms(TermAngleApprox<DEG>(L.c.a, L.c.b), px);
    }
    __syncthreads();
    if (mine) {  // field rows +k and -k of this pixel
      float d[ROW];
#pragma unroll
      for (int dx = -M; dx <= M; ++dx) {
        const int cq = c + dx;
        float v = 0.0f;
        if (k > 0 || dx > 0) {
          v = T[(dx + M) * NR + p];  // 0 when p + (k, dx) is outside
        } else if (dx < 0 && cq >= 0) {
          v = T[(-dx + M) * NR + p + dx];
        }
        d[dx + M] = v;
      }
      add_row(k, d);
      if (k > 0) {
        const int rq = r - k;
#pragma unroll
        for (int dx = -M; dx <= M; ++dx) {
          const int cq = c + dx;
          d[dx + M] = (rq >= 0 && cq >= 0 && cq < RX) ? T[(-dx + M) * NR + rq * RX + cq] : 0.0f;
        }
        add_row(-k, d);
      }
    }
    __syncthreads();  // T is rewritten by the next offset row
  }
  // window centred at region (r + ey, c + ex) = output (r + ey - R, c + ex - R)
  if (mine) {
#pragma unroll
    for (int ey = -R; ey <= R; ++ey)
#pragma unroll
      for (int ex = -R; ex <= R; ++ex) {
        const int oy = r + ey - R, ox = c + ex - R;
        if (oy >= 0 && oy < RTY && ox >= 0 && ox < kRTX) {
          const int j = (R - ey) * W + (R - ex);  // p's index in that window
          A[j * G::OUT + oy * kRTX + ox] = agg[ey + R][ex + R];
        }
      }
  }
  __syncthreads();
  reuse_finish<W, CRIT, APX, DEG, RTY, NT>(L, px, raw, A, x0, y0);
}

template <int W, int CRIT, int APX, int DEG, int RTY, int NT>
__device__ __forceinline__ void reuse_chunked_reg_tile(const Launch& L, int tile) {
  using G = ReuseGeom<W, RTY, NT>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
  TileSmem t;
  t.px = reinterpret_cast<float4*>(smem);
  t.raw = reinterpret_cast<uint32_t*>(smem + G::NR * 16);
  t.sw = G::RX;
  t.sh = G::RY;
  stage_tile<CRIT>(L, t, txi * kRTX, tyi * RTY, G::R);
  __syncthreads();
  reuse_chunked_reg_tile_body<W, CRIT, APX, DEG, RTY, NT>(L, tile);
}

// One 32 x 8 tile per CTA (a 256-thread CTA whose shared memory is reused:
// callers looping over tiles must __syncthreads() between calls).
template <int W, int CRIT, int APX, int DEG, int RTY = kRTY, int NT = kRTX * RTY>
__device__ __forceinline__ void reuse_any_tile(const Launch& L, int tile) {
  if (L.flags != nullptr) {  // uniform test
    if constexpr (W >= 7) {
      if (reuse_gated_skip_call<RTY, NT>(L, tile)) return;
    } else {
      if (reuse_gated_skip<RTY, NT>(L, tile)) return;
    }
  }
  if constexpr (W >= 7 && NT >= (kRTX + W - 1) * (RTY + W - 1)) {
    reuse_chunked_reg_tile<W, CRIT, APX, DEG, RTY, NT>(L, tile);
  } else if constexpr (W >= 7) {
    static_assert(RTY == kRTY && NT == kRTX * kRTY, "the chunked form has 32 x 8 tiles");
    reuse_chunked_tile<W, CRIT, APX, DEG>(L, tile);
  } else {
    reuse_tile<W, CRIT, APX, DEG, RTY, NT>(L, tile);
  }
}

// Persistent form of the tall tiles (one thread per region pixel, w <= 5):
// each CTA loops over tiles blockIdx.x, + gridDim.x, ...; while a tile's
// phases run, the next tile's region pixels are copied by cp.async into a
// spare buffer after the tile's shared memory (each thread the pixel it
// stages), so that staging waits on no global load.  32-bit pixels only.
// Gated form: a tile none of whose outputs is flagged is copied from the
// staged region (the others read the flags in the finish phase).
__host__ __device__ constexpr size_t reuse_persistent_smem_bytes(int w, int rty) {
  return reuse_smem_bytes(w, rty) + (size_t)(kRTX + w - 1) * (rty + w - 1) * 4;
}

template <int W, int CRIT, int APX, int DEG, int RTY, int NT>
__device__ __forceinline__ void reuse_tiles_persistent(const Launch& L, int ntiles) {
  using G = ReuseGeom<W, RTY, NT>;
  constexpr int R = G::R, RX = G::RX, NR = G::NR;
  static_assert(NT >= NR && W <= 5, "tall tiles, one thread per region pixel");
  extern __shared__ __align__(16) unsigned char smem[];
  float4* px = reinterpret_cast<float4*>(smem);
  uint32_t* raw = reinterpret_cast<uint32_t*>(smem + NR * 16);
  uint32_t* next = reinterpret_cast<uint32_t*>(smem + reuse_smem_bytes(W, RTY));
  const int p = threadIdx.x;
  const int ry = p / RX, rx = p - ry * RX;
  auto prefetch = [&](int tile) {
    if (p < NR) {
      const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
      const int gy = min(max(tyi * RTY + ry - R, 0), L.height - 1);
      const int gx = min(max(txi * kRTX + rx - R, 0), L.width - 1);
      const uint8_t* src = L.in + (long long)gy * L.in_pitch + 4LL * gx;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(next + p)),
                   "l"(src)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  int tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile);
  for (; tile < ntiles; tile += gridDim.x) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (p < NR) {  // the pixel this thread fetched
      const uint32_t v = next[p];
      raw[p] = v;
      px[p] = stage_cell<CRIT>(v);
    }
    const int tyi = tile / L.tiles_x, txi = tile - tyi * L.tiles_x;
    const int x0 = txi * kRTX, y0 = tyi * RTY;
    const int ox = p % kRTX, oy = p / kRTX;
    const bool out = p < G::OUT && x0 + ox < L.width && y0 + oy < L.height;
    bool skip = false;
    if (L.flags != nullptr) {  // gated form: a tile without a flag is copied whole
      const bool f = out && L.flags[(long long)(y0 + oy) * L.flag_pitch + x0 + ox] != 0;
      skip = !__syncthreads_or(f);  // also the barrier after staging
    } else {
      __syncthreads();  // the region is staged; `next` is free again
    }
    if (tile + (int)gridDim.x < ntiles) prefetch(tile + gridDim.x);
    if (skip) {
      if (out) store_px(L, x0 + ox, y0 + oy, raw[(oy + R) * RX + ox + R]);
      block_stats(L, out ? 1 : 0, 0, 0);
    } else {
      reuse_tile_body<W, CRIT, APX, DEG, RTY, NT>(L, tile);
    }
    __syncthreads();  // the finish phase's reads are done before the next staging
  }
}

inline size_t reuse_any_smem_bytes(int w, int rty = kRTY) {
  if (w >= 7) return rty == kRTY ? reuse_chunked_smem_bytes(w) : reuse_chunked_reg_smem_bytes(w, rty);
  return reuse_smem_bytes(w, rty);
}

// 32 x RTY outputs per CTA of NT threads: two 256-thread CTAs per SM at
// RTY = 8; one CTA of a thread per region pixel for taller tiles (a larger
// term table, fewer region pixels per output, phases in whole rounds)
template <int W, int CRIT, int APX, int DEG, int RTY, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1)
    reuse_kernel(const __grid_constant__ Launch L) {
  pdl_begin();
  if (L.gate_count != nullptr && *L.gate_count <= L.gate_limit) return;  // the sparse form ran
  reuse_any_tile<W, CRIT, APX, DEG, RTY, NT>(L, blockIdx.x);
}

// The persistent tall-tile form (32-bit pixels)
template <int W, int CRIT, int APX, int DEG, int RTY, int NT>
__global__ void __launch_bounds__(NT, 1)
    reuse_persistent_kernel(const __grid_constant__ Launch L, int ntiles) {
  pdl_begin();
  if (L.gate_count != nullptr && *L.gate_count <= L.gate_limit) return;  // the sparse form ran
  reuse_tiles_persistent<W, CRIT, APX, DEG, RTY, NT>(L, ntiles);
}

template <int W, int CRIT, int APX, int DEG, int RTY = reuse_tile_rows(W, CRIT),
          int NT = reuse_threads(W, RTY)>
cudaError_t launch_reuse_one(const Launch& L, int grid, cudaStream_t s) {
  // (7 x 7: the loop around the 49 register window sums spills; one tile per
  // CTA measured faster, 4.82 against 5.43 ms at 4096^2)
  if constexpr (W <= 5 && NT >= (kRTX + W - 1) * (RTY + W - 1)) {
    if (L.vec4_in) {
      const size_t smem = reuse_persistent_smem_bytes(W, RTY);
      auto kern = reuse_persistent_kernel<W, CRIT, APX, DEG, RTY, NT>;
      // resident CTAs of the whole device, found once per device (the
      // attribute set with it)
      static int resident[16] = {};
      int dev = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e != cudaSuccess) return e;
      int& res = resident[dev & 15];
      if (res == 0) {
        int sms = 0, per_sm = 0;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
        if (e != cudaSuccess) return e;
        res = std::max(per_sm, 1) * sms;
      }
      return launch_maybe_pdl(L.pdl != 0, kern, dim3(std::min(grid, res)), dim3(NT), smem, s, L,
                              grid);
    }
  }
  const size_t smem = reuse_any_smem_bytes(W, RTY);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(reuse_kernel<W, CRIT, APX, DEG, RTY, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return launch_maybe_pdl(L.pdl != 0, reuse_kernel<W, CRIT, APX, DEG, RTY, NT>, dim3(grid),
                          dim3(NT), smem, s, L);
}



// BVDF and EVBDF: exact or polynomial angle
template <int W, int CRIT>
cudaError_t launch_reuse_angle(const Launch& L, int apx, int degree, int grid, cudaStream_t s) {
  if (apx == kExact) return launch_reuse_one<W, CRIT, kExact, 0>(L, grid, s);
  switch (degree) {
    case 2: return launch_reuse_one<W, CRIT, kPoly, 2>(L, grid, s);
    case 3: return launch_reuse_one<W, CRIT, kPoly, 3>(L, grid, s);
    case 4: return launch_reuse_one<W, CRIT, kPoly, 4>(L, grid, s);
    case 5: return launch_reuse_one<W, CRIT, kPoly, 5>(L, grid, s);
    case 6: return launch_reuse_one<W, CRIT, kPoly, 6>(L, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

// VMF, BVDF and EVBDF
template <int W>
cudaError_t launch_reuse_sel(const Launch& L, int crit, int apx, int degree, int grid,
                             cudaStream_t s) {
  if (crit == kVMF) return launch_reuse_one<W, kVMF, kExact, 0>(L, grid, s);
  if (crit == kBVDF) return launch_reuse_angle<W, kBVDF>(L, apx, degree, grid, s);
  if (crit == kEVBDF) return launch_reuse_angle<W, kEVBDF>(L, apx, degree, grid, s);
  return cudaErrorInvalidValue;
}

template <int W, int CRIT>
cudaError_t launch_reuse_amnf_c(const Launch& L, int apx, int degree, int grid, cudaStream_t s) {
  if (apx == kExact) return launch_reuse_one<W, CRIT, kExact, 0>(L, grid, s);
  if (apx == kRational) return launch_reuse_one<W, CRIT, kRational, 4>(L, grid, s);
  switch (degree) {
    case 2: return launch_reuse_one<W, CRIT, kPoly, 2>(L, grid, s);
    case 3: return launch_reuse_one<W, CRIT, kPoly, 3>(L, grid, s);
    case 4: return launch_reuse_one<W, CRIT, kPoly, 4>(L, grid, s);
    case 5: return launch_reuse_one<W, CRIT, kPoly, 5>(L, grid, s);
    case 6: return launch_reuse_one<W, CRIT, kPoly, 6>(L, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

// AMNFE and AMNFG
template <int W>
cudaError_t launch_reuse_amnf(const Launch& L, int crit, int apx, int degree, int grid,
                              cudaStream_t s) {
  if (crit == kAMNFE) return launch_reuse_amnf_c<W, kAMNFE>(L, apx, degree, grid, s);
  if (crit == kAMNFG) return launch_reuse_amnf_c<W, kAMNFG>(L, apx, degree, grid, s);
  return cudaErrorInvalidValue;
}

// EVMF: the ENT function exact, polynomial or rational, as for AMNF's EXP
template <int W>
cudaError_t launch_reuse_evmf(const Launch& L, int apx, int degree, int grid, cudaStream_t s) {
  return launch_reuse_amnf_c<W, kEVMF>(L, apx, degree, grid, s);
}

}  // namespace vf
