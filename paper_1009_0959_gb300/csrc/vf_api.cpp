// vf_api.cpp -- the C ABI of include/vfilt.h: argument checks, the minimax
// coefficient cache and kernel dispatch.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>

#include "../../include/vfilt.h"
#include "vf_internal.h"

using namespace vf;

namespace {

// The paper's (4,4) minimax rationals (increasing powers), the library's own
// copy: Sec. 3.2, tab_exp_rat (exp(-z) on [0, 10]) and Sec. 3.3, tab_ent_rat
// (z ln z on [0.05, 1]).
const double kExpRatNum[5] = {3.206619e-02, -1.195191e-02, 1.756974e-03, -1.199261e-04,
                              3.182685e-06};
const double kExpRatDen[5] = {3.206627e-02, 2.011147e-02, 5.853684e-03, 9.780143e-04,
                              1.251598e-04};
const double kExpRatEps = 2.227050e-06;
const double kEntRatNum[5] = {-1.519742e-04, -6.835769e-02, -8.856923e-01, -5.369609e-01,
                              1.491165};
const double kEntRatDen[5] = {1.532270e-02, 3.987796e-01, 1.461793, 6.827004e-01,
                              -4.469776e-02};
const double kEntRatEps = 7.342477e-07;

struct FitKey {
  int kind;  // 0 polynomial, 1 (degree, degree) rational
  int fn, degree;
  double lo, hi;
  bool operator<(const FitKey& o) const {
    return std::tie(kind, fn, degree, lo, hi) < std::tie(o.kind, o.fn, o.degree, o.lo, o.hi);
  }
};
struct FitVal {
  double coef[8];  // polynomial, or the rational's numerator
  double den[8];   // rational denominator (den[0] = 1)
  double eps;
};

}  // namespace

struct vf_ctx {
  std::map<FitKey, FitVal> fits;
  // vf_set_coefficients: the caller's approximants, keyed (kind: 0 polynomial,
  // 1 rational; function; degree); they take the place of the library's fits
  // on every interval
  std::map<std::tuple<int, int, int>, FitVal> user;
  std::string last_error;
  int tile_rows = 4;  // TY of the per-window single-image launches
  int pair_reuse = 1;  // 0 never, 1 where it pays (BVDF, EVBDF), 2 always
  int gate_tc = 1;     // gate inference: 0 CUDA cores, 1 tcgen05, 2 warp-level mma
  int overlap = 1;     // programmatic dependent launches for vf_filter
  int gated_sparse = 200;  // vf_filter_gated: sparse form up to this many flagged per mille
  int* d_glist = nullptr;  // its pixel list and counter
  unsigned* d_gcount = nullptr;
  size_t glist_cap = 0;
  // device staging of vf_filter_host (grown on demand, freed by vf_destroy)
  uint8_t* d_stage = nullptr;
  size_t stage_bytes = 0;
  int stage_device = -1;
  // vf_filter_host_async: staging slots, each with its own stream
  struct HostSlot {
    uint8_t* d_buf = nullptr;
    size_t bytes = 0;
    int device = -1;
    cudaStream_t stream = nullptr;
    cudaEvent_t start = nullptr;  // orders the slot's work after the caller's stream
  };
  HostSlot slots[VF_HOST_SLOTS];
  int next_slot = 0;
};

namespace {

vf_status fail(vf_ctx* ctx, vf_status s, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return s;
}

const FitVal* user_fit(const vf_ctx* ctx, int kind, int fn, int degree) {
  auto it = ctx->user.find(std::make_tuple(kind, fn, degree));
  return it == ctx->user.end() ? nullptr : &it->second;
}

const FitVal* get_fit(vf_ctx* ctx, int fn, int degree, double lo, double hi) {
  if (const FitVal* u = user_fit(ctx, 0, fn, degree)) return u;
  FitKey k{0, fn, degree, lo, hi};
  auto it = ctx->fits.find(k);
  if (it != ctx->fits.end()) return &it->second;
  FitVal v{};
  if (!remez_fit(fn, degree, lo, hi, v.coef, &v.eps)) return nullptr;
  return &(ctx->fits[k] = v);
}

// The library's own best (degree, degree) rational of function fn on [lo, hi].
const FitVal* get_rational_fit(vf_ctx* ctx, int fn, int degree, double lo, double hi) {
  if (const FitVal* u = user_fit(ctx, 1, fn, degree)) return u;
  FitKey k{1, fn, degree, lo, hi};
  auto it = ctx->fits.find(k);
  if (it != ctx->fits.end()) return &it->second;
  FitVal v{};
  if (!remez_rational_fit(fn, degree, degree, lo, hi, v.coef, v.den, &v.eps)) return nullptr;
  return &(ctx->fits[k] = v);
}

float default_ent_cutoff(int n) { return n <= 9 ? 0.05f : 0.05f * 9.0f / (float)n; }

bool overlap(const uint8_t* a, size_t na, const uint8_t* b, size_t nb) {
  return a < b + nb && b < a + na;
}

}  // namespace

extern "C" {

vf_status vf_create(vf_ctx** ctx) {
  if (!ctx) return VF_ERR_ARG;
  *ctx = alloc_refused() ? nullptr : new (std::nothrow) vf_ctx();
  if (!*ctx) return VF_ERR_OOM;
  // the exact angle's arctangent polynomial, fitted once per context so that
  // every exact angle call (the allocation-free one included) finds it
  if (!get_fit(*ctx, VF_FN_HALF_ANGLE, kHalfAngleDegree, 0.0, 1.0)) {
    delete *ctx;
    *ctx = nullptr;
    return VF_ERR_ARG;
  }
  return VF_OK;
}

void vf_destroy(vf_ctx* ctx) {
  if (!ctx) return;
  if (ctx->d_stage) cudaFree(ctx->d_stage);
  if (ctx->d_glist) cudaFree(ctx->d_glist);
  if (ctx->d_gcount) cudaFree(ctx->d_gcount);
  for (auto& sl : ctx->slots) {
    if (sl.stream) {
      cudaStreamSynchronize(sl.stream);
      cudaStreamDestroy(sl.stream);
    }
    if (sl.start) cudaEventDestroy(sl.start);
    if (sl.d_buf) cudaFree(sl.d_buf);
  }
  delete ctx;
}

const char* vf_status_string(vf_status s) {
  switch (s) {
    case VF_OK: return "ok";
    case VF_ERR_ARG: return "invalid argument";
    case VF_ERR_ALIAS: return "input and output overlap";
    case VF_ERR_UNSUPPORTED: return "unsupported combination";
    case VF_ERR_CUDA: return "CUDA error";
    case VF_ERR_TIMEOUT: return "device wait timed out";
    case VF_ERR_OOM: return "out of memory";
  }
  return "unknown status";
}

const char* vf_last_error(const vf_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

vf_status vf_set_option(vf_ctx* ctx, vf_option opt, int value) {
  if (!ctx) return VF_ERR_ARG;
  switch (opt) {
    case VF_OPT_PAIR_REUSE:
      if (value < 0 || value > 2) return fail(ctx, VF_ERR_ARG, "pair reuse 0, 1 or 2");
      ctx->pair_reuse = value;
      return VF_OK;
    case VF_OPT_GATE_TENSOR_CORES:
      if (value < 0 || value > 2) return fail(ctx, VF_ERR_ARG, "gate tensor cores 0, 1 or 2");
      ctx->gate_tc = value;
      return VF_OK;
    case VF_OPT_OVERLAP_LAUNCH: ctx->overlap = value != 0; return VF_OK;
    case VF_OPT_GATED_SPARSE:
      if (value < 0 || value > 1000) return fail(ctx, VF_ERR_ARG, "gated sparse 0 .. 1000");
      ctx->gated_sparse = value;
      return VF_OK;
    case VF_OPT_TILE_ROWS:
      if (value != 2 && value != 4 && value != 8) return fail(ctx, VF_ERR_ARG, "tile rows 2, 4 or 8");
      ctx->tile_rows = value;
      return VF_OK;
  }
  return fail(ctx, VF_ERR_ARG, "unknown option");
}

void vf_default_params(vf_params* p) {
  if (!p) return;
  p->window = 3;
  p->criterion = VF_VMF;
  p->approx = VF_EXACT;
  p->degree = 4;
  p->precision = VF_FP32;
  p->kappa = 0.33f;
  p->exp_cutoff = 10.0f;
  p->ent_cutoff = -1.0f;
}

vf_status vf_get_approximant(vf_ctx* ctx, vf_function fn, vf_approx approx, int degree, double lo,
                             double hi, double* num, int* num_len, double* den, int* den_len,
                             double* eps) {
  if (!ctx || !num || !num_len || !den || !den_len || !eps) return VF_ERR_ARG;
  if (approx == VF_MINIMAX_RATIONAL) {
    if (fn != VF_FN_EXP && fn != VF_FN_ENT)
      return fail(ctx, VF_ERR_UNSUPPORTED, "the paper gives rationals for EXP and ENT only");
    const double* n = fn == VF_FN_EXP ? kExpRatNum : kEntRatNum;
    const double* d = fn == VF_FN_EXP ? kExpRatDen : kEntRatDen;
    for (int k = 0; k < 5; ++k) num[k] = n[k], den[k] = d[k];
    *num_len = 5;
    *den_len = 5;
    *eps = fn == VF_FN_EXP ? kExpRatEps : kEntRatEps;
    return VF_OK;
  }
  if (approx == VF_MINIMAX_RATIONAL_FIT) {
    if (degree < 2 || degree > 4) return fail(ctx, VF_ERR_ARG, "rational degree must be 2..4");
    if ((int)fn < 0 || (int)fn > 4 || !(hi > lo)) return fail(ctx, VF_ERR_ARG, "bad function/interval");
    const FitVal* f = get_rational_fit(ctx, (int)fn, degree, lo, hi);
    if (!f) return fail(ctx, VF_ERR_ARG, "rational minimax fit failed (pole on the interval)");
    for (int k = 0; k <= degree; ++k) num[k] = f->coef[k], den[k] = f->den[k];
    *num_len = degree + 1;
    *den_len = degree + 1;
    *eps = f->eps;
    return VF_OK;
  }
  if (approx != VF_MINIMAX_POLY) return fail(ctx, VF_ERR_ARG, "approx must be poly or rational");
  if (degree < 2 || degree > 7) return fail(ctx, VF_ERR_ARG, "degree must be 2..7");
  if ((int)fn < 0 || (int)fn > 4 || !(hi > lo)) return fail(ctx, VF_ERR_ARG, "bad function/interval");
  const FitVal* f = get_fit(ctx, (int)fn, degree, lo, hi);
  if (!f) return fail(ctx, VF_ERR_ARG, "minimax fit failed");
  for (int k = 0; k <= degree; ++k) num[k] = f->coef[k];
  *num_len = degree + 1;
  *den_len = 0;
  *eps = f->eps;
  return VF_OK;
}

vf_status vf_set_coefficients(vf_ctx* ctx, vf_function fn, vf_approx approx, int degree,
                              const double* num, int num_len, const double* den, int den_len,
                              double lo, double hi) {
  if (!ctx) return VF_ERR_ARG;
  if ((int)fn < 0 || (int)fn > 3)
    return fail(ctx, VF_ERR_ARG, "bad function (the exact angle's polynomial is fixed)");
  if (approx == VF_MINIMAX_RATIONAL)
    return fail(ctx, VF_ERR_UNSUPPORTED,
                "the paper's printed rationals are fixed; load a rational as "
                "VF_MINIMAX_RATIONAL_FIT");
  if (approx != VF_MINIMAX_POLY && approx != VF_MINIMAX_RATIONAL_FIT)
    return fail(ctx, VF_ERR_ARG, "approx must be VF_MINIMAX_POLY or VF_MINIMAX_RATIONAL_FIT");
  const int kind = approx == VF_MINIMAX_POLY ? 0 : 1;
  if (kind == 0 && (degree < 2 || degree > 6)) return fail(ctx, VF_ERR_ARG, "degree must be 2..6");
  if (kind == 1 && (degree < 2 || degree > 4))
    return fail(ctx, VF_ERR_ARG, "rational degree must be 2..4");
  const auto key = std::make_tuple(kind, (int)fn, degree);
  if (!num && num_len == 0 && !den && den_len == 0) {  // back to the library's own fit
    ctx->user.erase(key);
    return VF_OK;
  }
  if (!num || num_len != degree + 1)
    return fail(ctx, VF_ERR_ARG, "num must hold degree + 1 coefficients");
  if (kind == 0 && den_len != 0) return fail(ctx, VF_ERR_ARG, "a polynomial has no denominator");
  if (kind == 1 && (!den || den_len != degree + 1))
    return fail(ctx, VF_ERR_ARG, "den must hold degree + 1 coefficients");
  if (!std::isfinite(lo) || !std::isfinite(hi) || !(hi > lo))
    return fail(ctx, VF_ERR_ARG, "bad interval");
  FitVal v{};
  for (int k = 0; k < num_len; ++k) {
    if (!std::isfinite(num[k])) return fail(ctx, VF_ERR_ARG, "non-finite coefficient");
    v.coef[k] = num[k];
  }
  for (int k = 0; k < den_len; ++k) {
    if (!std::isfinite(den[k])) return fail(ctx, VF_ERR_ARG, "non-finite coefficient");
    v.den[k] = den[k];
  }
  if (!approximant_error((int)fn, v.coef, num_len, v.den, den_len, lo, hi, &v.eps))
    return fail(ctx, VF_ERR_ARG, "the denominator vanishes on the interval");
  ctx->user[key] = v;
  return VF_OK;
}

vf_status vf_row_quantum(vf_ctx* ctx, const vf_params* p, int* rows) {
  if (!ctx) return VF_ERR_ARG;
  if (!p || !rows) return fail(ctx, VF_ERR_ARG, "null pointer");
  if ((int)p->criterion < 0 || (int)p->criterion > 5 || (int)p->precision < 0 ||
      (int)p->precision > 2)
    return fail(ctx, VF_ERR_ARG, "bad enum");
  if (p->window != 3 && p->window != 5 && p->window != 7)
    return fail(ctx, VF_ERR_UNSUPPORTED, "windows 3, 5 and 7 are built");
  const int w = p->window, crit = (int)p->criterion;
  if (p->precision != VF_FP32) {
    *rows = ctx->tile_rows;  // packed tiles: 64 x TY outputs, one row per thread row
  } else if (use_pair_reuse(ctx, w, crit)) {
    *rows = reuse_tile_rows(w, crit);
  } else if (crit == kEVMF && w == 5) {
    *rows = evmf_queue_rows(w);  // the work-queue kernel's own tiles
  } else {
    *rows = ctx->tile_rows * outputs_per_thread(w, crit);
  }
  return VF_OK;
}

vf_status vf_band_plan(int height, int window, int quantum, int bands, int band, int* in_row0,
                       int* in_rows, int* out_row0, int* out_rows) {
  if (!in_row0 || !in_rows || !out_row0 || !out_rows) return VF_ERR_ARG;
  if (height < 1 || window < 1 || (window & 1) == 0 || quantum < 1 || bands < 1 ||
      bands > height || band < 0 || band >= bands)
    return VF_ERR_ARG;
  const int h = window / 2;
  const long long r0 = (long long)band * height / bands;
  const long long r1 = (long long)(band + 1) * height / bands;
  // the halo rows above, with the band's first row rounded down to the tile
  // quantum so that its tiles line up with the whole image's
  long long a = r0 - h;
  a = a <= 0 ? 0 : a / quantum * quantum;
  const long long b = std::min<long long>(height, r1 + h);
  *in_row0 = (int)a;
  *in_rows = (int)(b - a);
  *out_row0 = (int)r0;
  *out_rows = (int)(r1 - r0);
  return VF_OK;
}

}  // extern "C"

namespace vf {

vf_status prepare_launch(vf_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int height, int width,
                         int channels, size_t in_pitch, size_t out_pitch, const vf_params* p,
                         unsigned long long* d_stats, Launch* out, LaunchClass* cls) {
  if (!ctx) return VF_ERR_ARG;
  if (!d_in || !d_out || !p) return fail(ctx, VF_ERR_ARG, "null pointer");
  if (height < 1 || width < 1) return fail(ctx, VF_ERR_ARG, "image size must be >= 1 x 1");
  if (channels != 3 && channels != 4) return fail(ctx, VF_ERR_ARG, "channels must be 3 or 4");
  if (in_pitch < (size_t)width * channels || out_pitch < (size_t)width * channels)
    return fail(ctx, VF_ERR_ARG, "pitch smaller than a row");
  if ((int)p->criterion < 0 || (int)p->criterion > 5) return fail(ctx, VF_ERR_ARG, "bad criterion");
  if ((int)p->approx < 0 || (int)p->approx > 3) return fail(ctx, VF_ERR_ARG, "bad approximation");
  if ((int)p->precision < 0 || (int)p->precision > 2) return fail(ctx, VF_ERR_ARG, "bad precision");
  if (p->window < 1 || (p->window & 1) == 0 || p->window > 15)
    return fail(ctx, VF_ERR_ARG, "window must be odd, 1..15");
  if (p->window != 3 && p->window != 5 && p->window != 7)
    return fail(ctx, VF_ERR_UNSUPPORTED, "windows 3, 5 and 7 are built");
  if (p->approx == VF_MINIMAX_POLY && (p->degree < 2 || p->degree > 6))
    return fail(ctx, VF_ERR_ARG, "degree must be 2..6");
  if (p->approx == VF_MINIMAX_RATIONAL_FIT && (p->degree < 2 || p->degree > 4))
    return fail(ctx, VF_ERR_ARG, "rational degree must be 2..4");
  if (!(p->kappa >= 0.0f) || !(p->exp_cutoff > 0.0f)) return fail(ctx, VF_ERR_ARG, "bad kappa/cut-off");
  if (p->precision != VF_FP32 && p->criterion == VF_BVDF && p->approx != VF_MINIMAX_POLY)
    return fail(ctx, VF_ERR_UNSUPPORTED, "packed BVDF runs the minimax polynomial only");
  const size_t in_bytes = (size_t)(height - 1) * in_pitch + (size_t)width * channels;
  const size_t out_bytes = (size_t)(height - 1) * out_pitch + (size_t)width * channels;
  if (overlap(d_in, in_bytes, d_out, out_bytes))
    return fail(ctx, VF_ERR_ALIAS, "input and output overlap");

  const int w = p->window, n = w * w;
  const int crit = (int)p->criterion;
  // the library's own rational runs the rational kernels with its coefficients
  const bool rfit = p->approx == VF_MINIMAX_RATIONAL_FIT;
  int apx = rfit ? kRational : (int)p->approx;
  if (crit == kVMF) apx = kExact;  // the vector median has no elementary function
  if (apx == kRational && (crit == kBVDF || crit == kEVBDF))
    return fail(ctx, VF_ERR_UNSUPPORTED, "the paper gives no rational for arccos");
  if (crit == kEVBDF && p->precision != VF_FP32)
    return fail(ctx, VF_ERR_UNSUPPORTED, "EVBDF runs in FP32 only");

  Launch L{};
  L.in = d_in;
  L.out = d_out;
  L.height = height;
  L.width = width;
  L.channels = channels;
  L.vec4_in = channels == 4 && ((uintptr_t)d_in % 4 == 0) && in_pitch % 4 == 0;
  L.vec4_out = channels == 4 && ((uintptr_t)d_out % 4 == 0) && out_pitch % 4 == 0;
  L.in_pitch = (long long)in_pitch;
  L.out_pitch = (long long)out_pitch;
  L.kappa_scale = (float)std::pow((double)n, -(double)p->kappa / 3.0);
  L.exp_cutoff = p->exp_cutoff;
  L.ent_cutoff = p->ent_cutoff < 0.0f ? default_ent_cutoff(n) : p->ent_cutoff;
  L.stats = d_stats;
  L.pdl = ctx->overlap;

  // coefficients of the approximant, rounded to FP32, zero above the degree
  auto put = [](float* dst, const double* src, int len) {
    for (int k = 0; k < 8; ++k) dst[k] = k < len ? (float)src[k] : 0.0f;
  };
  if (apx == kExact && (crit == kBVDF || crit == kEVBDF)) {
    // the exact angle's arctangent polynomial (fitted when the context was made)
    const FitVal* f = get_fit(ctx, VF_FN_HALF_ANGLE, kHalfAngleDegree, 0.0, 1.0);
    if (!f) return fail(ctx, VF_ERR_ARG, "minimax fit failed");
    put(L.c.a, f->coef, kHalfAngleDegree + 1);
  }
  if (apx != kExact) {
    if (crit == kBVDF || crit == kEVBDF) {
      const FitVal* lo = get_fit(ctx, 0, p->degree, 0.0, 0.5);
      const FitVal* hi = get_fit(ctx, 1, p->degree, 0.0, 1.0 / std::sqrt(2.0));
      if (!lo || !hi) return fail(ctx, VF_ERR_ARG, "minimax fit failed");
      put(L.c.a, lo->coef, p->degree + 1);
      put(L.c.b, hi->coef, p->degree + 1);
      if (crit == kEVBDF) {  // the switch's ENT polynomial, same degree
        if (!(L.ent_cutoff > 0.0f) || L.ent_cutoff >= 1.0f)
          return fail(ctx, VF_ERR_ARG, "the ENT polynomial needs a cut-off in (0, 1)");
        const FitVal* f = get_fit(ctx, 3, p->degree, (double)L.ent_cutoff, 1.0);
        if (!f) return fail(ctx, VF_ERR_ARG, "minimax fit failed");
        put(L.c.e, f->coef, p->degree + 1);
      }
    } else if (crit == kAMNFE || crit == kAMNFG) {
      if (apx == kRational && rfit) {
        const FitVal* f = get_rational_fit(ctx, 2, p->degree, 0.0, (double)p->exp_cutoff);
        if (!f) return fail(ctx, VF_ERR_ARG, "rational minimax fit failed");
        put(L.c.a, f->coef, p->degree + 1);
        put(L.c.b, f->den, p->degree + 1);
      } else if (apx == kRational) {
        if (p->exp_cutoff != 10.0f)
          return fail(ctx, VF_ERR_UNSUPPORTED, "the paper's EXP rational is fitted on [0, 10]");
        put(L.c.a, kExpRatNum, 5);
        put(L.c.b, kExpRatDen, 5);
      } else {
        const FitVal* f = get_fit(ctx, 2, p->degree, 0.0, (double)p->exp_cutoff);
        if (!f) return fail(ctx, VF_ERR_ARG, "minimax fit failed");
        put(L.c.a, f->coef, p->degree + 1);
      }
    } else if (crit == kEVMF) {
      if (apx == kRational && rfit) {
        if (!(L.ent_cutoff > 0.0f) || L.ent_cutoff >= 1.0f)
          return fail(ctx, VF_ERR_ARG, "the ENT rational fit needs a cut-off in (0, 1)");
        const FitVal* f = get_rational_fit(ctx, 3, p->degree, (double)L.ent_cutoff, 1.0);
        if (!f) return fail(ctx, VF_ERR_ARG, "rational minimax fit failed");
        put(L.c.a, f->coef, p->degree + 1);
        put(L.c.b, f->den, p->degree + 1);
      } else if (apx == kRational) {
        put(L.c.a, kEntRatNum, 5);
        put(L.c.b, kEntRatDen, 5);
      } else {
        if (!(L.ent_cutoff > 0.0f) || L.ent_cutoff >= 1.0f)
          return fail(ctx, VF_ERR_ARG, "the ENT polynomial needs a cut-off in (0, 1)");
        const FitVal* f = get_fit(ctx, 3, p->degree, (double)L.ent_cutoff, 1.0);
        if (!f) return fail(ctx, VF_ERR_ARG, "minimax fit failed");
        put(L.c.a, f->coef, p->degree + 1);
      }
    }
  }
  *out = L;
  cls->crit = crit;
  cls->w = w;
  cls->apx = apx;
  cls->deg = apx == kPoly ? p->degree : (apx == kRational ? 4 : 0);
  cls->precision = (int)p->precision;
  return VF_OK;
}

vf_status set_error(vf_ctx* ctx, vf_status s, const char* msg) { return fail(ctx, s, msg); }

int gate_tensor_cores(const vf_ctx* ctx) { return ctx->gate_tc; }

bool use_pair_reuse(const vf_ctx* ctx, int w, int crit) {
  return ctx->pair_reuse == 2 ? has_reuse_kernel(w, crit)
                              : (ctx->pair_reuse == 1 && reuse_pays(w, crit));
}

const double* cached_fit(const vf_ctx* ctx, int fn, int degree, double lo, double hi) {
  if (const FitVal* u = user_fit(ctx, 0, fn, degree)) return u->coef;
  auto it = ctx->fits.find(FitKey{0, fn, degree, lo, hi});
  return it == ctx->fits.end() ? nullptr : it->second.coef;
}

bool cached_rational_fit(const vf_ctx* ctx, int fn, int degree, double lo, double hi,
                         const double** num, const double** den) {
  if (const FitVal* u = user_fit(ctx, 1, fn, degree)) {
    *num = u->coef;
    *den = u->den;
    return true;
  }
  auto it = ctx->fits.find(FitKey{1, fn, degree, lo, hi});
  if (it == ctx->fits.end()) return false;
  *num = it->second.coef;
  *den = it->second.den;
  return true;
}

void paper_rational(int fn, const double** num, const double** den) {
  *num = fn == 2 ? kExpRatNum : kEntRatNum;
  *den = fn == 2 ? kExpRatDen : kEntRatDen;
}

}  // namespace vf

extern "C" {

vf_status vf_filter(vf_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int height, int width,
                    int channels, size_t in_pitch, size_t out_pitch, const vf_params* p,
                    void* stream, unsigned long long* d_stats) {
  Launch L;
  LaunchClass cls;
  vf_status st = prepare_launch(ctx, d_in, d_out, height, width, channels, in_pitch, out_pitch, p,
                                d_stats, &L, &cls);
  if (st != VF_OK) return st;
  return launch_single(ctx, L, cls, (cudaStream_t)stream);
}

}  // extern "C"

namespace vf {

vf_status launch_single(vf_ctx* ctx, Launch L, const LaunchClass& cls, cudaStream_t s) {
  const int height = L.height, width = L.width;
  if (cls.precision == VF_FP32 && use_pair_reuse(ctx, cls.w, cls.crit)) {
    L.tiles_x = (width + kTX - 1) / kTX;
    const int rows = reuse_tile_rows(cls.w, cls.crit);
    const long long rgrid = (long long)L.tiles_x * ((height + rows - 1) / rows);
    if (rgrid > 0x7fffffffLL) return fail(ctx, VF_ERR_UNSUPPORTED, "image too large");
    cudaError_t e = launch_reuse(L, cls.crit, cls.w, cls.apx, cls.deg, (int)rgrid, s);
    if (e != cudaSuccess) return fail(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
    return VF_OK;
  }
  const int ty = ctx->tile_rows;  // thread rows of the CTA
  const int cols = cls.precision == VF_FP32 ? kTX : kPackedTileCols;
  const int rows = cls.precision == VF_FP32 ? ty * outputs_per_thread(cls.w, cls.crit) : ty;
  L.tiles_x = (width + cols - 1) / cols;
  const int tiles_y = (height + rows - 1) / rows;
  const long long grid = (long long)L.tiles_x * tiles_y;
  if (grid > 0x7fffffffLL) return fail(ctx, VF_ERR_UNSUPPORTED, "image too large");
  cudaError_t e = cls.precision == VF_FP32
                      ? launch_filter(L, cls.crit, cls.w, cls.apx, cls.deg, ty, (int)grid, s)
                      : launch_packed(L, cls.precision, cls.crit, cls.w, cls.apx, cls.deg, ty,
                                      (int)grid, s);
  if (e != cudaSuccess) return fail(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  return VF_OK;
}

int gated_sparse_permille(const vf_ctx* ctx) { return ctx->gated_sparse; }

vf_status gated_scratch(vf_ctx* ctx, size_t pixels, int** list, unsigned** count) {
  if (!ctx->d_gcount && device_alloc(&ctx->d_gcount, sizeof(unsigned)) != cudaSuccess) {
    ctx->d_gcount = nullptr;
    cudaGetLastError();
    return fail(ctx, VF_ERR_OOM, "gated list allocation failed");
  }
  if (pixels > ctx->glist_cap) {
    if (ctx->d_glist) {
      cudaDeviceSynchronize();  // earlier calls may still read the old list
      cudaFree(ctx->d_glist);
    }
    ctx->d_glist = nullptr;
    ctx->glist_cap = 0;
    if (device_alloc(&ctx->d_glist, pixels * sizeof(int)) != cudaSuccess) {
      ctx->d_glist = nullptr;
      cudaGetLastError();
      return fail(ctx, VF_ERR_OOM, "gated list allocation failed");
    }
    ctx->glist_cap = pixels;
  }
  *list = ctx->d_glist;
  *count = ctx->d_gcount;
  return VF_OK;
}

namespace {
// allocations left before the injected failure; < 0: disarmed
std::atomic<int> g_fail_after{-1};
}  // namespace

bool alloc_refused() {
  int k = g_fail_after.load();
  while (k >= 0) {
    if (g_fail_after.compare_exchange_weak(k, k - 1)) return k == 0;
  }
  return false;
}

}  // namespace vf

extern "C" {

int vf_debug_fail_alloc(int after) { return g_fail_after.exchange(after < 0 ? -1 : after); }

vf_status vf_filter_host(vf_ctx* ctx, const uint8_t* h_in, uint8_t* h_out, int height, int width,
                         int channels, size_t in_pitch, size_t out_pitch, const vf_params* p,
                         void* stream) {
  if (!ctx) return VF_ERR_ARG;
  if (!h_in || !h_out || !p) return fail(ctx, VF_ERR_ARG, "null pointer");
  if (height < 1 || width < 1) return fail(ctx, VF_ERR_ARG, "image size must be >= 1 x 1");
  if (channels != 3 && channels != 4) return fail(ctx, VF_ERR_ARG, "channels must be 3 or 4");
  const size_t row = (size_t)width * channels;
  if (in_pitch < row || out_pitch < row) return fail(ctx, VF_ERR_ARG, "pitch smaller than a row");
  const size_t dpitch = (row + 15) / 16 * 16;  // 16-byte rows on the device
  const size_t need = 2 * dpitch * (size_t)height;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  if (need > ctx->stage_bytes || dev != ctx->stage_device) {
    if (ctx->d_stage) cudaFree(ctx->d_stage);
    ctx->d_stage = nullptr;
    ctx->stage_bytes = 0;
    if (device_alloc(&ctx->d_stage, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, VF_ERR_OOM, "device staging allocation failed");
    }
    ctx->stage_bytes = need;
    ctx->stage_device = dev;
  }
  uint8_t* d_in = ctx->d_stage;
  uint8_t* d_out = ctx->d_stage + dpitch * (size_t)height;
  cudaStream_t s = (cudaStream_t)stream;
  e = cudaMemcpy2DAsync(d_in, dpitch, h_in, in_pitch, row, height, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  vf_status st = vf_filter(ctx, d_in, d_out, height, width, channels, dpitch, dpitch, p, stream,
                           nullptr);
  if (st != VF_OK) return st;
  e = cudaMemcpy2DAsync(h_out, out_pitch, d_out, dpitch, row, height, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  return VF_OK;
}

vf_status vf_filter_host_async(vf_ctx* ctx, const uint8_t* h_in, uint8_t* h_out, int height,
                               int width, int channels, size_t in_pitch, size_t out_pitch,
                               const vf_params* p, void* stream) {
  if (!ctx) return VF_ERR_ARG;
  if (!h_in || !h_out || !p) return fail(ctx, VF_ERR_ARG, "null pointer");
  if (height < 1 || width < 1) return fail(ctx, VF_ERR_ARG, "image size must be >= 1 x 1");
  if (channels != 3 && channels != 4) return fail(ctx, VF_ERR_ARG, "channels must be 3 or 4");
  const size_t row = (size_t)width * channels;
  if (in_pitch < row || out_pitch < row) return fail(ctx, VF_ERR_ARG, "pitch smaller than a row");
  const size_t dpitch = (row + 15) / 16 * 16;
  const size_t need = 2 * dpitch * (size_t)height;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  vf_ctx::HostSlot& sl = ctx->slots[ctx->next_slot];
  if (sl.stream && sl.device != dev) {  // slot made on another device: rebuild it here
    cudaStreamSynchronize(sl.stream);
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.start);
    cudaFree(sl.d_buf);
    sl = vf_ctx::HostSlot{};
  }
  if (!sl.stream) {
    if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&sl.start, cudaEventDisableTiming)) != cudaSuccess)
      return fail(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
    sl.device = dev;
  }
  if (need > sl.bytes) {  // grow: the slot's earlier work may still read the old buffer
    if ((e = cudaStreamSynchronize(sl.stream)) != cudaSuccess)
      return fail(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
    if (sl.d_buf) cudaFree(sl.d_buf);
    sl.d_buf = nullptr;
    sl.bytes = 0;
    if (device_alloc(&sl.d_buf, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, VF_ERR_OOM, "device staging allocation failed");
    }
    sl.bytes = need;
  }
  ctx->next_slot = (ctx->next_slot + 1) % VF_HOST_SLOTS;
  uint8_t* d_in = sl.d_buf;
  uint8_t* d_out = sl.d_buf + dpitch * (size_t)height;
  if ((e = cudaEventRecord(sl.start, (cudaStream_t)stream)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(sl.stream, sl.start, 0)) != cudaSuccess ||
      (e = cudaMemcpy2DAsync(d_in, dpitch, h_in, in_pitch, row, height, cudaMemcpyHostToDevice,
                             sl.stream)) != cudaSuccess)
    return fail(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  vf_status st = vf_filter(ctx, d_in, d_out, height, width, channels, dpitch, dpitch, p, sl.stream,
                           nullptr);
  if (st != VF_OK) return st;
  e = cudaMemcpy2DAsync(h_out, out_pitch, d_out, dpitch, row, height, cudaMemcpyDeviceToHost,
                        sl.stream);
  if (e != cudaSuccess) return fail(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  return VF_OK;
}

vf_status vf_host_sync(vf_ctx* ctx) {
  if (!ctx) return VF_ERR_ARG;
  vf_status st = VF_OK;
  for (auto& sl : ctx->slots) {
    if (!sl.stream) continue;
    cudaError_t e = cudaStreamSynchronize(sl.stream);
    if (e != cudaSuccess && st == VF_OK) st = fail(ctx, VF_ERR_CUDA, cudaGetErrorString(e));
  }
  return st;
}

}  // extern "C"
