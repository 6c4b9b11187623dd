// vf_internal.h -- types shared by the library's translation units (not part
// of the public ABI; include/vfilt.h is).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/vfilt.h"

namespace vf {

constexpr int kTX = 32;  // output pixels per tile row (one warp)
// Degree of the exact angle's arctangent polynomial (VF_FN_HALF_ANGLE): the
// kernels evaluate its kHalfAngleDegree + 1 = 8 coefficients, in Coeffs::a.
constexpr int kHalfAngleDegree = 7;

enum { kVMF = 0, kBVDF = 1, kAMNFE = 2, kAMNFG = 3, kEVMF = 4, kEVBDF = 5 };
enum { kExact = 0, kPoly = 1, kRational = 2 };

// Approximant coefficients rounded to FP32, increasing powers.
//   BVDF: a = arccos piece on [0, 0.5], b = 2 arcsin(tau/sqrt2) piece
//   AMNF / EVMF polynomial: a; rational: a = numerator, b = denominator
//   EVBDF: a, b the arccos pieces as for BVDF, e the ENT polynomial
struct Coeffs {
  float a[8];
  float b[8];
  float e[8];
};

// Everything a launch needs, passed by value as the kernel parameter.
struct Launch {
  const uint8_t* in;
  uint8_t* out;
  int height, width, channels;
  int vec4_in, vec4_out;  // 32-bit pixel loads / stores allowed
  long long in_pitch, out_pitch;
  int tiles_x;            // tiles per tile row
  float kappa_scale;      // n^(-kappa/3)
  float exp_cutoff;
  float ent_cutoff;
  Coeffs c;
  unsigned long long* stats;  // optional device counters
  int pdl;                    // launch as a programmatic dependent (host side)
  // gated form in the pair-reuse kernels: non-null = filter only the pixels
  // whose flag byte is non-zero, copy the others (null for every other call)
  const uint8_t* flags;
  long long flag_pitch;
  // the gated filter's tile forms when the sparse form may take the call: a
  // CTA returns at once if *gate_count <= gate_limit (null otherwise)
  const unsigned* gate_count;
  unsigned gate_limit;
};

// Register aggregates (fully unrolled pair loop) or shared-memory aggregate
// slots (rolled row-pair loop) for a window / criterion.
constexpr bool uses_reg_path(int w, int crit) {
  return w == 3 || (w == 5 && crit != kBVDF && crit != kEVBDF);
}

// Output rows per thread of the single-image per-window kernels: two for
// VMF and AMNF (two vertically adjacent windows share w(w - 1) samples and
// their pairs), one otherwise.
constexpr int outputs_per_thread(int w, int crit) {
  return (w <= 7 && (crit == kVMF || crit == kAMNFE || crit == kAMNFG)) ? 2 : 1;
}

// Shared memory bytes of one CTA of 32 x ty threads for window w (reg: the
// aggregates live in registers, no shared-memory slots).
inline size_t smem_bytes(int w, int crit, int ty, bool reg) {
  size_t sw = kTX + w - 1, sh = ty + w - 1, threads = (size_t)kTX * ty;
  size_t b = sw * sh * 20;
  if (!reg) b += (size_t)w * w * threads * 4;
  b += threads * 4;  // EVMF list
  return b;
}
inline size_t smem_bytes(int w, int crit, int ty) { return smem_bytes(w, crit, ty, uses_reg_path(w, crit)); }

// Per-(criterion, window) launchers, one translation unit each
// (vf_k_<criterion>_w<w>.cu).  Return the CUDA error of the launch
// (cudaErrorInvalidValue for a combination with no kernel).
#define VF_DECLARE_LAUNCH(name)                                                         \
  cudaError_t launch_##name##_w3(const Launch&, int, int, int, int, cudaStream_t);   \
  cudaError_t launch_##name##_w5(const Launch&, int, int, int, int, cudaStream_t);   \
  cudaError_t launch_##name##_w7(const Launch&, int, int, int, int, cudaStream_t);
VF_DECLARE_LAUNCH(vmf)
VF_DECLARE_LAUNCH(bvdf)
VF_DECLARE_LAUNCH(amnfe)
VF_DECLARE_LAUNCH(amnfg)
VF_DECLARE_LAUNCH(evmf)
VF_DECLARE_LAUNCH(evbdf)
#undef VF_DECLARE_LAUNCH

// Packed-precision launchers (vf_p_<fp16|bf16>_w<w>.cu); one CTA covers
// 64 x ty outputs.
#define VF_DECLARE_PACKED(name)                                                            \
  cudaError_t launch_packed_##name##_w3(const Launch&, int, int, int, int, int, cudaStream_t); \
  cudaError_t launch_packed_##name##_w5(const Launch&, int, int, int, int, int, cudaStream_t); \
  cudaError_t launch_packed_##name##_w7(const Launch&, int, int, int, int, int, cudaStream_t);
VF_DECLARE_PACKED(fp16)
VF_DECLARE_PACKED(bf16)
#undef VF_DECLARE_PACKED
constexpr int kPackedTileCols = 64;

// Pair-reuse launchers (vf_r_w<w>_<sel|amnf|evmf>.cu): one CTA covers 32 x
// RTY outputs; windows 3, 5 (whole term table) and 7 (table built one offset
// row at a time), every criterion in FP32.
constexpr int kReuseTileRows = 8;
// Output rows of a single-image pair-reuse tile: taller tiles for BVDF (and
// EVBDF, EVMF) 3 x 3 (14 rows), 5 x 5 (20 rows) and every 7 x 7 filter
// (16 rows), whose CTA has one thread
// per region pixel (34 x 16 = 544, 36 x 24 = 864, 38 x 22 = 836 -> 864):
// fewer region pixels per output (1.35 at w = 5 instead of 36 x 12 / 256 =
// 1.69), both phases in whole rounds and, at w = 5, 27 warps per SM instead
// of 16 (measured 5,350 / 9,278 Mpix/s for the exact / degree-4 5 x 5 filter
// against 3,681 / 6,801 with 32 x 8 tiles).  At w = 7 the thread keeps its
// pixel's 49 window sums in registers (3,188 / 3,606 Mpix/s at 4096^2
// against 1,791 for degree 4 with 32 x 8 tiles and shared-memory sums; 12
// rows 2,750 / 3,095, 20 rows spill and gain nothing).  8 otherwise; the
// batched kernel always uses 8.
constexpr int reuse_tile_rows(int w, int crit) {
  return w == 7 ? 16 : ((crit != kBVDF && crit != kEVBDF && crit != kEVMF) ? 8 : (w == 5 ? 20 : 14));
}
// Tile rows of the EVMF work-queue kernel (5 x 5): 8 at 5 x 5 (less halo per
// output, fuller batches; measured 4-13 % faster than 4; one CTA per SM of 16
// rows / 128 registers or 24 rows / 80 registers measured 5-12 % slower than
// three of 8 rows); 4 for larger windows.
constexpr int evmf_queue_rows(int w) { return w <= 5 ? 8 : 4; }
cudaError_t launch_reuse_sel_w3(const Launch&, int, int, int, int, cudaStream_t);
cudaError_t launch_reuse_sel_w5(const Launch&, int, int, int, int, cudaStream_t);
cudaError_t launch_reuse_amnf_w3(const Launch&, int, int, int, int, cudaStream_t);
cudaError_t launch_reuse_amnf_w5(const Launch&, int, int, int, int, cudaStream_t);
cudaError_t launch_reuse_sel_w7(const Launch&, int, int, int, int, cudaStream_t);
cudaError_t launch_reuse_amnf_w7(const Launch&, int, int, int, int, cudaStream_t);
cudaError_t launch_reuse_evmf_w3(const Launch&, int, int, int, cudaStream_t);
cudaError_t launch_reuse_evmf_w5(const Launch&, int, int, int, cudaStream_t);
cudaError_t launch_reuse_evmf_w7(const Launch&, int, int, int, cudaStream_t);
inline bool has_reuse_kernel(int w, int crit) { return w == 3 || w == 5 || w == 7; }
// Where the reuse kernels are the faster choice (measured on GB300 at
// 1024 x 1024): the angle terms (BVDF), 2.0 - 3.4x; for the cheap L2 / L1
// terms the table and box-sum traffic costs more than the terms it saves
// (EVMF 20.5k / 8.8k / 3.7k Mpix/s at w = 3 / 5 / 7 against 32.1k / 9.7k /
// 3.7k for the per-window kernels and the work queue; AMNF 7 x 7 4.4k against
// 6.5k; VMF 7 x 7 5.5k against 5.3k, within the noise).
inline bool reuse_pays(int w, int crit) {
  return has_reuse_kernel(w, crit) && (crit == kBVDF || crit == kEVBDF);
}
cudaError_t launch_reuse(const Launch& L, int crit, int w, int apx, int degree, int grid,
                         cudaStream_t s);

// Dispatch on criterion and window (vf_dispatch.cpp).
cudaError_t launch_filter(const Launch& L, int criterion, int w, int approx, int degree, int ty,
                          int grid, cudaStream_t s);
// precision 1 = FP16x2, 2 = BF16x2
cudaError_t launch_packed(const Launch& L, int precision, int criterion, int w, int approx,
                          int degree, int ty, int grid, cudaStream_t s);

// The kernel class of a request: criterion, window, approximation, degree.
struct LaunchClass {
  int crit, w, apx, deg, precision;
};

// Argument checks, coefficients and the Launch block of one image (shared by
// vf_filter and the batched calls).  d_stats may be null.
vf_status prepare_launch(vf_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int height, int width,
                         int channels, size_t in_pitch, size_t out_pitch, const vf_params* p,
                         unsigned long long* d_stats, Launch* out, LaunchClass* cls);

// The launch of vf_filter for a prepared image: the pair-reuse, per-window or
// packed kernel the context's options select, on stream s.
vf_status launch_single(vf_ctx* ctx, Launch L, const LaunchClass& cls, cudaStream_t s);

// Gate inference engine (context option): 0 CUDA cores, 1 tcgen05, 2 mma.sync.
int gate_tensor_cores(const vf_ctx* ctx);
// VF_OPT_GATED_SPARSE (per mille of the pixels) and the sparse form's scratch:
// a list of H x W pixel indices and its counter (grown on demand, VF_ERR_OOM)
int gated_sparse_permille(const vf_ctx* ctx);
vf_status gated_scratch(vf_ctx* ctx, size_t pixels, int** list, unsigned** count);

// Whether an FP32 call of window w and criterion crit runs the pair-reuse
// kernels under the context's VF_OPT_PAIR_REUSE setting.
bool use_pair_reuse(const vf_ctx* ctx, int w, int crit);

// Record an error text in the context and return s.
vf_status set_error(vf_ctx* ctx, vf_status s, const char* msg);

// Coefficients of a fit already in the context's cache, or null; never fits
// or allocates.
const double* cached_fit(const vf_ctx* ctx, int fn, int degree, double lo, double hi);
// The same for the library's (degree, degree) rational fits.
bool cached_rational_fit(const vf_ctx* ctx, int fn, int degree, double lo, double hi,
                         const double** num, const double** den);

// The paper's (4,4) rationals (fn 2: exp(-z), fn 3: z ln z), 5 coefficients each.
void paper_rational(int fn, const double** num, const double** den);

// Host Remez exchange (FP64) of the library: minimax polynomial of degree
// `degree` for function id (0 acos, 1 2 asin(t/sqrt2), 2 exp(-z), 3 z ln z)
// on [lo, hi]; coefficients in increasing powers of the argument.
bool remez_fit(int fn, int degree, double lo, double hi, double* coef, double* eps);

// Host rational Remez (FP64, Sec. 2, the class R^n_m): the best p/q with
// deg p <= m, deg q <= n for function id fn on [lo, hi]; monomial
// coefficients num[0..m], den[0..n] with den[0] = 1.  False when the exchange
// meets a denominator with a zero on [lo, hi].
bool remez_rational_fit(int fn, int m, int n, double lo, double hi, double* num, double* den,
                        double* eps);

// Maximum error of p/q (q = 1 when den_len = 0) against function id fn on a
// 20,001-point grid of [lo, hi]; false when the denominator changes sign or
// vanishes on the grid.
bool approximant_error(int fn, const double* num, int num_len, const double* den, int den_len,
                       double lo, double hi, double* eps);

// Failure injection (vf_debug_fail_alloc): true when the armed countdown
// reaches this allocation, which the caller then treats as out of memory.
bool alloc_refused();

// cudaMalloc through the failure-injection countdown.
template <class T>
cudaError_t device_alloc(T** p, size_t bytes) {
  if (alloc_refused()) return cudaErrorMemoryAllocation;
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

}  // namespace vf
