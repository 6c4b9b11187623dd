/*
 * vfilt.h -- C ABI of the GB300 (sm_103a) vector order-statistic filters.
 *
 * The library computes, for every pixel of an M x N RGB image, the output
 * y(r,c) = F(W(r,c)) of a filter F over the w x w window W(r,c) that slides
 * over the image in raster order (arXiv 1009.0959, Sec. 3).  F is one of
 *   VF_VMF    vector median: argmin_i sum_j ||x_i - x_j||_2
 *             (Sec. 3.3, first branch of Eq. equ_evf)
 *   VF_BVDF   basic vector directional filter: argmin_i sum_j A(x_i, x_j),
 *             A = arccos of the normalised dot product (Sec. 3.1)
 *   VF_AMNFE  adaptive multichannel non-parametric filter, exponential
 *             kernel exp(-||x||_1)                  (Sec. 3.2, Eq. equ_amnf)
 *   VF_AMNFG  the same with the Gaussian kernel exp(-0.5 ||x||_2^2)
 *   VF_EVMF   entropy vector median filter: VMF where P_C > beta_C, the
 *             centre elsewhere                      (Sec. 3.3, Eq. equ_evf)
 * with the elementary function of the criterion (arccos, exp, z log z)
 * evaluated exactly (CUDA's single-precision math library) or through a
 * minimax polynomial of degree 2..6 (Sec. 2, Tables 1-2) or the paper's (4,4)
 * minimax rationals (Sec. 3.2 tab_exp_rat, Sec. 3.3 tab_ent_rat).
 *
 * Conventions shared by every call:
 *   - Images are interleaved 8-bit, 3 (RGB) or 4 (RGBX) bytes per pixel,
 *     rows `pitch` bytes apart.  Only the first three bytes are colour; a
 *     fourth byte is copied from the centre pixel (AMNF) or the selected
 *     pixel (selection filters).
 *   - Borders replicate the nearest image pixel; the window samples are
 *     indexed in raster order, argmin ties go to the lowest index.
 *   - Device pointers are owned by the caller.  The library never frees or
 *     retains caller memory after a call returns.  Input and output must not
 *     overlap (the windows read neighbours): VF_ERR_ALIAS.
 *   - Calls are asynchronous on the given stream (0 = legacy default stream)
 *     and return a status; they never abort.  A CUDA launch error is
 *     VF_ERR_CUDA and its text is kept in the context (vf_last_error).
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef VFILT_H
#define VFILT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VF_OK = 0,
  VF_ERR_ARG = 1,         /* null pointer, bad size, bad enum value */
  VF_ERR_ALIAS = 2,       /* input and output ranges overlap */
  VF_ERR_UNSUPPORTED = 3, /* valid request this build does not provide */
  VF_ERR_CUDA = 4,        /* a CUDA call failed (text in vf_last_error) */
  VF_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  VF_ERR_OOM = 6          /* device or host allocation failed */
} vf_status;

/* VF_EVBDF: the generalised entropy vector filter of Sec. 3.3 with the angle
 * of Sec. 3.1 as its distance: EVMF's switch (P_C > beta_C), BVDF's selection
 * in the switched windows, the centre elsewhere.  VF_EXACT or
 * VF_MINIMAX_POLY (one degree for the arccos pieces and the ENT
 * polynomial); single-image FP32 calls only (vf_filter, vf_filter_host). */
typedef enum {
  VF_VMF = 0,
  VF_BVDF = 1,
  VF_AMNFE = 2,
  VF_AMNFG = 3,
  VF_EVMF = 4,
  VF_EVBDF = 5
} vf_criterion;

/* VF_MINIMAX_RATIONAL: the paper's printed (4,4) rationals (EXP and ENT);
 * VF_MINIMAX_RATIONAL_FIT: the library's own best (d,d) rational, d = degree
 * in 2..4, fitted on the filter's interval ([0, exp_cutoff] for EXP,
 * [ent_cutoff, 1] for ENT) by a rational Remez exchange (Sec. 2, the class
 * R^n_m). */
typedef enum {
  VF_EXACT = 0,
  VF_MINIMAX_POLY = 1,
  VF_MINIMAX_RATIONAL = 2,
  VF_MINIMAX_RATIONAL_FIT = 3
} vf_approx;

/* Arithmetic of the pairwise terms and of the approximant evaluation.  The
 * aggregates are always accumulated in FP32. */
typedef enum { VF_FP32 = 0, VF_FP16X2 = 1, VF_BF16X2 = 2 } vf_precision;

/* Elementary functions the minimax approximants stand in for. */
typedef enum {
  VF_FN_ACOS_LO = 0, /* arccos(z) on [0, 0.5]                    (Table 1, ARCCOS) */
  VF_FN_ACOS_HI = 1, /* 2 arcsin(tau / sqrt 2) on [0, 1/sqrt 2]   (Table 1, ARCSIN) */
  VF_FN_EXP = 2,     /* exp(-z) on [0, exp_cutoff]                (Table 2)         */
  VF_FN_ENT = 3,     /* z ln z on [ent_cutoff, 1]                 (tab_ent_rat)     */
  VF_FN_HALF_ANGLE = 4 /* 2 atan(sqrt s) / sqrt s on [0, 1]: not in the paper; the
                          exact angle A = u P(u^2), u = tan(A/2) = |a x b| /
                          (|a||b| + a.b), with P of degree 7 (read-only)     */
} vf_function;

/* Filter parameters.  Fill with vf_default_params, then override. */
typedef struct {
  int window;             /* w: 3, 5 or 7 (n = w*w samples)                  */
  vf_criterion criterion;
  vf_approx approx;       /* VF_EXACT for VF_VMF (it has no elementary fn)   */
  int degree;             /* polynomial degree 2..6 (VF_MINIMAX_POLY)        */
  vf_precision precision;
  float kappa;            /* AMNF kernel-width exponent; Sec. 3.2: 0.33      */
  float exp_cutoff;       /* exp(-z) = 0 for z > exp_cutoff; Sec. 3.2: 10    */
  float ent_cutoff;       /* z ln z = 0 for z < ent_cutoff; Sec. 3.3: 0.05 at
                             n = 9.  A negative value selects the default
                             0.05 * 9 / n for n > 9 (0.05 at n = 9).          */
} vf_params;

/* Optional per-call counters, accumulated (atomically) into a caller-owned
 * DEVICE array of three unsigned long long: [0] pixels written,
 * [1] near ties (selection filters: best and second-best aggregate of a
 * different colour within 1e-5 relative; EVMF: also a switch decision within
 * 1e-5 relative), [2] EVMF pixels sent to the vector median. */
#define VF_STAT_PIXELS 0
#define VF_STAT_NEAR_TIES 1
#define VF_STAT_SWITCHED 2

typedef struct vf_ctx vf_ctx;

/* Create / destroy a context.  It holds the fitted coefficient cache (the
 * exact angle's arctangent polynomial is fitted on creation, a few
 * milliseconds of host work), the last error text and the device scratch of
 * the batched calls. */
vf_status vf_create(vf_ctx** ctx);
void vf_destroy(vf_ctx* ctx);

const char* vf_status_string(vf_status s);
const char* vf_last_error(const vf_ctx* ctx);

/* Context options (execution choices; results agree within the parity bar).
 *   VF_OPT_PAIR_REUSE  pair-reuse kernels (each pairwise term computed once
 *                      per 32 x 8 tile (BVDF, EVBDF and EVMF 3 x 3: 32 x 14,
 *                      5 x 5: 32 x 20; every 7 x 7 filter: 32 x 16) and
 *                      shared by every window holding the pair), for every
 *                      FP32 criterion with 3 x 3, 5 x 5 and 7 x 7 windows:
 *                      0 never (per-window kernels), 1 where they are faster
 *                      (default: BVDF and EVBDF), 2 always.
 *   VF_OPT_TILE_ROWS   thread rows TY of the per-window kernels' CTAs: 2, 4
 *                      (default) or 8 (32 x TY outputs; 32 x 2TY for VMF
 *                      and AMNF with w <= 5, whose threads filter two
 *                      windows; the EVMF work-queue kernel picks its own).
 *   VF_OPT_GATE_TENSOR_CORES  the engine of vf_gate_infer: 1 (default) the
 *                      three convolutions on the 5th-generation tensor cores
 *                      (tcgen05 MMAs with TMEM accumulators over rows of 128
 *                      cells, a layer's three tap rows side by side in one
 *                      MMA's N dimension); 2 the warp-level mma
 *                      instructions of earlier tensor cores; both with BF16
 *                      operands (activations rounded to BF16 between layers)
 *                      and FP32 accumulation; 0: CUDA cores with FP32
 *                      activations.
 *   VF_OPT_OVERLAP_LAUNCH  1 (default): vf_filter's kernels are launched as
 *                      programmatic dependents of the previous kernel in the
 *                      stream: their CTAs may be scheduled while that kernel
 *                      drains, and wait for its completion (and the
 *                      visibility of its memory) before their first access
 *                      to device memory, so stream order is kept; 0: plain
 *                      launches.
 *   VF_OPT_GATED_SPARSE  vf_filter_gated's sparse form, in flagged pixels per
 *                      mille (0 .. 1000): a first kernel copies the
 *                      unflagged pixels and lists the flagged ones, a second
 *                      filters the listed pixels one window each; when the
 *                      list holds more than that many per mille of the
 *                      pixels, the tile form runs instead (the choice is made
 *                      on the device, from the list's length: no host
 *                      synchronisation).  Default 200 (the sparse form at
 *                      up to 20 % flagged pixels; measured faster than the
 *                      tile forms below about 22 % for the 5 x 5 BVDF);
 *                      0: the tile form only; 1000: the sparse form only. */
typedef enum {
  VF_OPT_PAIR_REUSE = 0,
  VF_OPT_TILE_ROWS = 1,
  VF_OPT_GATE_TENSOR_CORES = 2,
  VF_OPT_OVERLAP_LAUNCH = 3,
  VF_OPT_GATED_SPARSE = 4
} vf_option;
vf_status vf_set_option(vf_ctx* ctx, vf_option opt, int value);

/* window 3, VF_VMF, VF_EXACT, degree 4, FP32, kappa 0.33, exp_cutoff 10,
 * ent_cutoff -1 (the window's default). */
void vf_default_params(vf_params* p);

/* The minimax approximant the library evaluates for `fn` (Sec. 2): for
 * VF_MINIMAX_POLY the library's own Remez exchange fit (host, FP64) of degree
 * `degree` on [lo, hi]; for VF_MINIMAX_RATIONAL the paper's printed (4,4)
 * rational (VF_FN_EXP: tab_exp_rat on [0, 10]; VF_FN_ENT: tab_ent_rat on
 * [0.05, 1]; lo and hi are ignored); for VF_MINIMAX_RATIONAL_FIT the
 * library's own best (degree, degree) rational on [lo, hi] (degree 2..4,
 * denominator normalised to den[0] = 1).  Polynomial degrees 2..7 (the
 * filters evaluate 2..6; VF_FN_HALF_ANGLE with degree 7 on [0, 1] is the
 * polynomial of the exact angle, fitted when the context is created).  num[0..*num_len), den[0..*den_len)
 * receive coefficients in increasing powers (den_len = 0 for a polynomial;
 * arrays of 8 suffice), *eps the maximum error on [lo, hi] (fits) or on the
 * printed rational's interval (its printed value).  Fits are cached in the
 * context.  Host memory; synchronous.
 * Errors: VF_ERR_ARG (null pointers, bad enum, degree or interval; a fit
 * whose denominator vanishes on the interval), VF_ERR_UNSUPPORTED (a printed
 * rational for a function the paper gives none for). */
vf_status vf_get_approximant(vf_ctx* ctx, vf_function fn, vf_approx approx, int degree,
                             double lo, double hi, double* num, int* num_len, double* den,
                             int* den_len, double* eps);

/* Load the caller's own approximant of `fn` into the context (Sec. 2: any
 * minimax polynomial or rational the caller fitted, e.g. the coefficients
 * printed in Table 1 (VF_FN_ACOS_LO / VF_FN_ACOS_HI, degree 4) or Table 2
 * (VF_FN_EXP, degrees 2..4)).
 *   approx    VF_MINIMAX_POLY (degree 2..6): num[0..degree] in increasing
 *             powers, den NULL and den_len 0; or VF_MINIMAX_RATIONAL_FIT
 *             (degree 2..4): num[0..degree] / den[0..degree]
 *   lo, hi    the interval the coefficients are meant for; the library
 *             measures their maximum error against the function there (on
 *             a 20,001-point grid) and reports it through vf_get_approximant
 * From then on every call in this context that evaluates the degree-`degree`
 * approximant of that kind for `fn` uses these coefficients (rounded to
 * FP32 for the kernels) in place of the library's own fit, whatever the
 * filter's interval or cut-off: vf_filter, vf_filter_host(_async),
 * vf_filter_gated, vf_batch_create (a batch keeps the coefficients it was
 * created with) and vf_batch_run_static.  vf_get_approximant returns them as
 * given.  num = NULL, num_len = 0, den = NULL, den_len = 0 removes them (the
 * library's fit is used again).  Host memory, read during the call;
 * synchronous; no device work.
 * Errors: VF_ERR_ARG (null context, bad enum (VF_FN_HALF_ANGLE included: the
 * exact angle's polynomial is fixed), degree or interval, wrong coefficient
 * counts, a non-finite coefficient, a denominator with a zero or
 * a sign change on [lo, hi]), VF_ERR_UNSUPPORTED (VF_MINIMAX_RATIONAL: the
 * paper's printed rationals are fixed). */
vf_status vf_set_coefficients(vf_ctx* ctx, vf_function fn, vf_approx approx, int degree,
                              const double* num, int num_len, const double* den, int den_len,
                              double lo, double hi);

/* Filter one image (Sec. 3): d_out(r,c) = F(W(r,c)) for every pixel.
 *   d_in, d_out   device pointers, height x width pixels of `channels`
 *                 (3 or 4) bytes, rows in_pitch / out_pitch bytes apart
 *                 (pitch >= width * channels)
 *   p             filter parameters (host memory, read during the call)
 *   stream        CUDA stream (cudaStream_t) the kernel is launched on
 *   d_stats       optional device counters (see VF_STAT_*), or NULL; when
 *                 given, the kernel also detects near ties (a little slower)
 * The call only enqueues work on `stream`: with VF_OPT_OVERLAP_LAUNCH (the
 * default) the kernel is a programmatic dependent of the stream's previous
 * kernel and waits for it before reading d_in, so stream order holds.
 * Errors: VF_ERR_ARG (null pointers, sizes < 1, channels not 3/4, pitch too
 * small, bad enums, degree out of 2..6 (2..4 for VF_MINIMAX_RATIONAL_FIT), a
 * failed minimax fit), VF_ERR_ALIAS, VF_ERR_UNSUPPORTED (window not 3/5/7, a
 * rational for BVDF or EVBDF, the printed EXP rational with a cut-off other
 * than 10, FP16X2/BF16X2 for a criterion without a packed path), VF_ERR_CUDA. */
vf_status vf_filter(vf_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int height, int width,
                    int channels, size_t in_pitch, size_t out_pitch, const vf_params* p,
                    void* stream, unsigned long long* d_stats);

/* The same filter on HOST images: copies h_in to device staging owned by the
 * context (allocated on first use, grown when a larger image comes, freed by
 * vf_destroy), runs vf_filter there and copies the result to h_out, all on
 * `stream`, then waits for the stream.  Pinned host memory (cudaHostAlloc)
 * makes the copies asynchronous DMA; pageable memory works too.  h_in and
 * h_out may be the same buffer (the device copies are distinct).
 * Errors: as vf_filter, plus VF_ERR_OOM when the staging cannot be
 * allocated.  Synchronous with respect to the host. */
vf_status vf_filter_host(vf_ctx* ctx, const uint8_t* h_in, uint8_t* h_out, int height, int width,
                         int channels, size_t in_pitch, size_t out_pitch, const vf_params* p,
                         void* stream);

/* Pipelined host-buffer filtering for many images: the same work as
 * vf_filter_host, but the call returns once the copies and the kernel are
 * enqueued.  The context keeps VF_HOST_SLOTS staging slots, each with its
 * own stream (non-blocking, created on first use); consecutive calls take the
 * slots in turn, so the copies of one image overlap the filtering of the
 * others.  A call starts after the work enqueued on `stream` before it (an
 * event); it reads h_in and writes h_out asynchronously, so both must stay
 * valid and h_in unchanged until vf_host_sync returns.  Host memory must be
 * pinned (cudaHostAlloc / cudaHostRegister) for the overlap.
 * Errors: as vf_filter_host; an error of an enqueued copy or kernel is
 * reported by vf_host_sync. */
#define VF_HOST_SLOTS 6
vf_status vf_filter_host_async(vf_ctx* ctx, const uint8_t* h_in, uint8_t* h_out, int height,
                               int width, int channels, size_t in_pitch, size_t out_pitch,
                               const vf_params* p, void* stream);

/* Waits until every vf_filter_host_async call of the context has completed
 * (its output is in host memory).  VF_ERR_CUDA if one of them failed. */
vf_status vf_host_sync(vf_ctx* ctx);

/* ---- row bands: one image split over several devices or calls --------------
 * Every output pixel depends only on its own window (Sec. 3: y(r,c) =
 * F(W(r,c))), so an image can be filtered in horizontal bands, each band a
 * separate vf_filter call (on its own GPU, or one after another) on a copy of
 * its rows plus (w - 1) / 2 halo rows above and below.  The band calls give
 * the whole-image call's bytes when each band's first row lines up with the
 * kernel's output tiles: vf_row_quantum gives that row quantum and
 * vf_band_plan rounds the band's first input row down to it.
 *
 * vf_row_quantum: output rows per tile of the kernel vf_filter launches for
 * `p` with this context's options (*rows).  Host only.
 * Errors: VF_ERR_ARG (null pointers, bad enums), VF_ERR_UNSUPPORTED (window
 * not 3/5/7). */
vf_status vf_row_quantum(vf_ctx* ctx, const vf_params* p, int* rows);

/* vf_band_plan: band `band` of `bands` (0-based) of an image `height` rows
 * high, window `window`: the band's output rows are [*out_row0, *out_row0 +
 * *out_rows) = [band * height / bands, (band + 1) * height / bands) (integer
 * division); its input is the *in_rows image rows from *in_row0 on: the
 * output rows, (window - 1) / 2 halo rows below (fewer at the image's bottom)
 * and the halo above, extended up to a multiple of `quantum` (0 at the
 * top).  vf_filter on those input rows (as an image of *in_rows rows) gives
 * the band's output rows at rows *out_row0 - *in_row0 onwards of its output.
 * Host arithmetic only; no context needed.
 * Errors: VF_ERR_ARG (null pointers, height < 1, an even or non-positive
 * window, quantum < 1, bands < 1 or > height, band outside [0, bands)). */
vf_status vf_band_plan(int height, int window, int quantum, int bands, int band, int* in_row0,
                       int* in_rows, int* out_row0, int* out_rows);

/* ---- batched form: many images in one persistent launch ------------------ */

/* One image of a batch: device buffers (caller-owned, as in vf_filter) and its
 * own filter parameters (window, criterion, approximation, degree...). */
typedef struct {
  const uint8_t* d_in;
  uint8_t* d_out;
  int height, width, channels;
  size_t in_pitch, out_pitch;
  vf_params params;
} vf_image_desc;

typedef struct vf_batch vf_batch;

/* Validate `count` descriptors (each as vf_filter would; the first failure is
 * returned) and build the work queue: all 32 x TY output tiles of all images,
 * images ordered by decreasing cost per tile, with their approximant
 * coefficients, copied to device memory that the batch owns (freed by
 * vf_batch_destroy).  Synchronous.  The batch keeps the device pointers: the
 * images must stay allocated while the batch is launched.
 * Errors: those of vf_filter, VF_ERR_ARG for count < 1, VF_ERR_OOM. */
vf_status vf_batch_create(vf_ctx* ctx, const vf_image_desc* descs, int count, vf_batch** batch);

/* Filter every image of the batch on `stream`: with VF_BATCH_ONE_KERNEL (the
 * default) ONE persistent kernel of SMs x CTAs-per-SM CTAs pulls tiles from a
 * device counter (reset by a memset on the same stream) until the queue is
 * empty; with VF_BATCH_CLASS_KERNELS one such kernel per image class on the
 * batch's branch streams (see vf_batch_set_mode).  Asynchronous; may be
 * captured into a CUDA graph by the caller.  Launches of one batch on
 * different streams must not overlap (they share the counters). */
vf_status vf_batch_launch(vf_batch* b, void* stream);

/* The same launch as a CUDA graph (memset node + kernel node), instantiated
 * on the first call (and after vf_batch_autotune / vf_batch_configure) and
 * replayed with cudaGraphLaunch on `stream`. */
vf_status vf_batch_graph_launch(vf_batch* b, void* stream);

/* Autotuner: times every tile shape (32 x TY thread rows, TY = 2, 4, 8) and
 * pixels-per-thread setting (see vf_batch_set_pixels_per_thread) with every
 * resident CTA count (1 .. occupancy maximum) on the batch itself, and the
 * class-kernel form (vf_batch_set_mode) (one warm-up and three timed
 * launches each, CUDA events on `stream`), keeps the fastest and reports it
 * (any out pointer may be NULL; the pixels per thread through
 * vf_batch_get_config, the form through vf_batch_get_mode).  Synchronous;
 * writes the outputs (the same values each time). */
vf_status vf_batch_autotune(vf_batch* b, void* stream, int* tile_rows, int* ctas_per_sm,
                            float* best_ms);

/* Set the configuration of the one-kernel form by hand (and select that
 * form): tile_rows 2, 4 or 8; ctas_per_sm 0 (the occupancy maximum) up to
 * that maximum.  Synchronous; not while a launch of the batch is in flight. */
vf_status vf_batch_configure(vf_batch* b, int tile_rows, int ctas_per_sm);

/* Pixels per thread of the VMF and AMNF tiles with 3 x 3 and 5 x 5 windows:
 * 1 (one window per thread, 32 x TY output tiles), 2 (two vertically
 * adjacent windows per thread sharing their common samples' pairs, 32 x 2TY
 * tiles), or 0 (the default: 2 for AMNF and 3 x 3 VMF, 1 for 5 x 5 VMF,
 * whose two-window body needs more registers than the shared kernel has).
 * Other images always take one window per thread.  Selects the one-kernel
 * form.  Synchronous; not while a launch of the batch is in flight. */
vf_status vf_batch_set_pixels_per_thread(vf_batch* b, int pixels_per_thread);

/* Execution form of the batch:
 *   VF_BATCH_ONE_KERNEL     one persistent kernel runs the tiles of every
 *                           image (the default; configured by the calls above)
 *   VF_BATCH_CLASS_KERNELS  one persistent kernel per image class (window x
 *                           criterion x approximation), each with the tile
 *                           shape, block size and shared memory of that
 *                           class's single-image kernel (two windows per
 *                           thread for VMF / AMNF, the tall pair-reuse tiles
 *                           for BVDF, the work queue for EVMF 5 x 5 and
 *                           per-window tiles for the other EVMF windows), or,
 *                           for a class where that is faster, one
 *                           single-image launch per image (BVDF by default);
 *                           the classes run concurrently on the batch's own
 *                           branch streams, forked from and joined to the
 *                           caller's stream (one CUDA graph with
 *                           vf_batch_graph_launch), costliest class first.
 * vf_batch_autotune times, per class, its class kernel against its
 * single-image launches and keeps the faster, then times both forms and keeps
 * the faster.  Synchronous; not while a launch of the batch is in flight. */
#define VF_BATCH_ONE_KERNEL 0
#define VF_BATCH_CLASS_KERNELS 1
vf_status vf_batch_set_mode(vf_batch* b, int mode);
vf_status vf_batch_get_mode(const vf_batch* b, int* mode);

/* The current configuration (any out pointer may be NULL). */
vf_status vf_batch_get_config(const vf_batch* b, int* tile_rows, int* ctas_per_sm,
                              int* pixels_per_thread);

void vf_batch_destroy(vf_batch* b);

/* ---- allocation-free batched call ------------------------------------------
 * No counterpart in the paper.  For callers that must not allocate GPU memory
 * while they filter: for example a real-time video pipeline, or a plug-in in a
 * host application that reserves all device memory up front, where cudaMalloc
 * on the frame path is forbidden because it can stall the whole device and its
 * latency has no bound.  vf_batch_run_static filters up to
 * VF_STATIC_MAX_IMAGES images exactly as vf_batch_create + vf_batch_launch
 * would (same kernel, 32 x 4 tiles, the occupancy maximum of resident CTAs)
 * but keeps its scratch (tile counter, tile table, image descriptors) in one
 * fixed device array inside the library (about 40 KB) instead of memory it
 * allocates.  Every GPU that loads the library holds that array until the
 * process exits.  The caller still passes the input and output images.
 *   - The first call on a device looks the array's address up on that device
 *     (with the device current); make that first call before any stream
 *     capture.
 *   - Calls share the one array and it keeps the last call's contents: each
 *     call resets the counter itself, but calls whose work overlaps on the GPU
 *     (different streams, no ordering between them) race and corrupt each
 *     other.  Calls on one stream are ordered and safe.
 *   - Nothing is fitted here: a polynomial approximant must already be in the
 *     context's cache (any earlier vf_filter, vf_batch_create or
 *     vf_get_approximant call in the same context with the same criterion,
 *     degree and cut-offs puts it there); otherwise VF_ERR_UNSUPPORTED.
 *   - No error text is recorded in the context (that could allocate).
 *   - The H2D copies of the descriptors come from the library's own static
 *     host buffer; the host side of the calls is serialised by a mutex.
 *     Because a replay of a recorded copy would read that buffer again after
 *     later calls changed it, a call on a stream that is being captured is
 *     refused with VF_ERR_UNSUPPORTED.
 * Errors: VF_ERR_ARG (null pointers, count < 1, bad sizes or enums, an
 * ENT cut-off outside (0, 1) for a fitted ENT approximant),
 * VF_ERR_UNSUPPORTED (count > VF_STATIC_MAX_IMAGES, a window other than
 * 3/5/7, a precision other than FP32, an approximant not yet fitted, a
 * capturing stream), VF_ERR_ALIAS, VF_ERR_CUDA (the runtime's last error is
 * cleared before returning).
 * Asynchronous on `stream` apart from the pageable descriptor copies. */
#define VF_STATIC_MAX_IMAGES 256
vf_status vf_batch_run_static(vf_ctx* ctx, const vf_image_desc* descs, int count, void* stream);

/* ---- learned impulse gate (not in the paper) --------------------------------
 * A small convolutional detector that decides which pixels get the window
 * filter, as the EVMF switch (Sec. 3.3, Eq. equ_evf) decides it with an
 * entropy test.  Network: x0 = RGB / 255 - 1/2; z1 = conv3x3(x0) (16 channels),
 * ReLU; z2 = conv3x3 (16 -> 16), ReLU; z3 = conv3x3 (16 -> 1); p = sigmoid(z3);
 * zero padding at every layer.  Parameters: a flat FP32 vector of
 * VF_GATE_NPARAM values in the order W1[16][3][3][3], b1[16],
 * W2[16][16][3][3], b2[16], W3[1][16][3][3], b3[1].  The kernels use BF16
 * copies of the weights with FP32 activations and accumulation; training
 * updates FP32 master weights with Adam (beta1 0.9, beta2 0.999, eps 1e-8)
 * on the mean binary cross-entropy against 0/1 targets.  Training is
 * deterministic (no floating-point atomics): the same seed, data and steps
 * give the same bits, also across vf_gate_save / vf_gate_load. */
#define VF_GATE_NPARAM 2913

typedef struct vf_gate vf_gate;

/* New gate with He-normal weights drawn from `seed` (zero biases) and zeroed
 * Adam state; device memory owned by the gate.  Synchronous. */
vf_status vf_gate_create(vf_ctx* ctx, unsigned long long seed, vf_gate** gate);
/* Host FP32 parameters in / out (n must be VF_GATE_NPARAM).  Setting resets
 * the Adam state and the step count.  Synchronous. */
vf_status vf_gate_set_params(vf_gate* g, const float* params, int n);
vf_status vf_gate_get_params(vf_gate* g, float* params, int n);

/* Batch of `count` equally sized images (device, 3 or 4 bytes per pixel, rows
 * `pitch` bytes apart, image k starting at d_imgs + k * height * pitch) with
 * 0/1 targets (device bytes, count x height x width, dense).
 *   vf_gate_gradient    writes the gradient of the mean BCE to d_grad
 *                       (VF_GATE_NPARAM floats, device), the loss to d_loss
 *                       and the probabilities to d_prob (count x H x W
 *                       floats); any of the three may be NULL
 *   vf_gate_train_step  the same forward / backward, then one Adam step with
 *                       learning rate lr; d_loss (device float) may be NULL
 * Asynchronous on `stream`.  The gate keeps activation scratch sized for the
 * largest batch seen (VF_ERR_OOM if it cannot grow). */
vf_status vf_gate_gradient(vf_gate* g, const uint8_t* d_imgs, const uint8_t* d_targets, int count,
                           int height, int width, int channels, size_t pitch, float* d_grad,
                           float* d_loss, float* d_prob, void* stream);
vf_status vf_gate_train_step(vf_gate* g, const uint8_t* d_imgs, const uint8_t* d_targets,
                             int count, int height, int width, int channels, size_t pitch,
                             float lr, float* d_loss, void* stream);

/* Fused inference over one image: d_flags[y * flag_pitch + x] = 1 where the
 * impulse probability exceeds `threshold` (0 < threshold < 1), else 0; d_prob
 * (height x width floats, dense) receives the probabilities.  Either output
 * may be NULL (not both).  Asynchronous on `stream`. */
vf_status vf_gate_infer(vf_gate* g, const uint8_t* d_in, int height, int width, int channels,
                        size_t pitch, float threshold, uint8_t* d_flags, size_t flag_pitch,
                        float* d_prob, void* stream);

/* vf_filter restricted to the pixels whose flag byte is non-zero; all other
 * pixels are copied from d_in.  VMF, BVDF, AMNFE and AMNFG in FP32 (EVMF has
 * its own switch: VF_ERR_UNSUPPORTED).  Otherwise as vf_filter; the third
 * counter (VF_STAT_SWITCHED) counts the flagged pixels.  Two forms, chosen
 * on the device under VF_OPT_GATED_SPARSE from the number of flags:
 *   tile form    where vf_filter runs the pair-reuse kernels
 *                (VF_OPT_PAIR_REUSE) so does this call, with the same sums
 *                (tiles without a flag are copied whole), else the
 *                per-window kernels on each tile's flagged pixels; a flagged
 *                pixel gets vf_filter's output
 *   sparse form  the flagged pixels are listed and each is filtered with its
 *                own window by the per-window kernels' code (the bytes of
 *                the tile form with VF_OPT_PAIR_REUSE = 0); it can differ
 *                from vf_filter's output only where two aggregates lie
 *                within rounding of each other (near ties).
 * Uses a pixel list in the context's scratch (grown on demand: VF_ERR_OOM). */
vf_status vf_filter_gated(vf_ctx* ctx, const uint8_t* d_in, uint8_t* d_out, int height, int width,
                          int channels, size_t in_pitch, size_t out_pitch, const uint8_t* d_flags,
                          size_t flag_pitch, const vf_params* p, void* stream,
                          unsigned long long* d_stats);

/* Checkpoint: magic "VFGATE01", version 1, VF_GATE_NPARAM, step, seed,
 * FP32 master weights, Adam first and second moments, CRC-32 of all that.
 * Load restores weights, moments, step and seed (VF_ERR_ARG on a bad file
 * or CRC).  Synchronous. */
vf_status vf_gate_save(vf_gate* g, const char* path);
vf_status vf_gate_load(vf_gate* g, const char* path);
unsigned long long vf_gate_step_count(const vf_gate* g);
/* Whether every tensor-core inference since the last check completed: the
 * tcgen05 engine waits for its MMAs with a bounded wait (about a second);
 * if one gave up, that launch skipped its remaining tiles and set a flag in
 * the gate.  Waits for the device (synchronous), returns VF_ERR_TIMEOUT (and
 * clears the flag) if a wait gave up, else VF_OK. */
vf_status vf_gate_check(vf_gate* g);
void vf_gate_destroy(vf_gate* g);

/* ---- failure injection (tests) ------------------------------------------- */

/* Makes an allocation of this library fail on purpose, so that the error
 * paths can be exercised without exhausting memory: after `after` further
 * allocations succeed, the next one fails as if the memory were exhausted
 * (VF_ERR_OOM from the call that made it) and the hook disarms itself;
 * after < 0 disarms it at once.  Counted allocations: the handles of
 * vf_create, vf_batch_create and vf_gate_create, and every device buffer the
 * library allocates (host staging, batch descriptors, gate weights and
 * training scratch).  A failed call releases what it had allocated and
 * leaves the context usable.  Process-wide; returns the previous setting. */
int vf_debug_fail_alloc(int after);

#ifdef __cplusplus
}
#endif

#endif /* VFILT_H */
