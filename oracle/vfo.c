/*
 * vfo.c -- plain, slow, FP64 CPU oracle of the sliding-window vector
 * order-statistic filters of Celebi, Kingravi, Lukac and Celiker,
 * "Cost-Effective Implementation of Order-Statistics Based Vector Filters
 * Using Minimax Approximations" (arXiv 1009.0959).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the test suite, the package's smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no header, helper or
 * table with the CUDA path: the approximant coefficients it evaluates are
 * handed in by the Python side of the oracle (oracle/remez.py,
 * oracle/paper_tables.py).
 *
 * Every step follows the paper's definitions, one window at a time, in the
 * paper's order, without any blocking or reuse:
 *   Sec. 3 (problem statement): an M x N image of RGB vectors; a w x w window
 *     W(r,c) slides in raster order; y(r,c) = F(W(r,c)); the window samples
 *     are re-indexed x_1..x_n in raster order, the centre is x_{(n+1)/2}.
 *   Sec. 3.1, BVDF equation: y = argmin_i sum_j A(x_i,x_j), A = arccos of the
 *     normalised dot product; the arccos identity for z >= 0.5 and the
 *     tau = sqrt(1-z) substitution of Table 1.
 *   Sec. 3.2, Eq. (equ_amnf): kernel-density weighted mean with widths
 *     h_i = n^(-kappa/3) sum_j ||x_i-x_j||_1, kernels exp(-||.||_1) (AMNFE)
 *     and exp(-0.5||.||_2^2) (AMNFG); EXP cut-off T: 0 outside [0,T].
 *   Sec. 3.3, Eq. (equ_evf): EVMF switch P_C > beta_C between the vector
 *     median (first branch = the VMF) and the identity; ENT(z) = z log z with
 *     cut-off T: 0 below T.
 *
 * Readings where the paper is silent (all documented in the design notes):
 *   - borders replicate the nearest image pixel (clamp-to-edge);
 *   - the self term j = i is skipped (it is 0 for the exact functions and the
 *     same constant for every i under an approximation);
 *   - argmin ties go to the lowest raster index;
 *   - a pair involving a zero vector has cosine 0 (angle pi/2);
 *   - constant windows (all h_i = 0, or sum_j r_j = 0) output the centre;
 *   - AMNF outputs are rounded half-to-even and clamped to [0,255];
 *   - the EXP and ENT cut-offs are part of the functions for the exact and
 *     the approximate variants alike (Sec. 3.2 - 3.3 motivate them by the
 *     behaviour of the functions themselves).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* criterion codes (mirrored by the Python wrapper, not shared with CUDA) */
enum { VFO_VMF = 0, VFO_BVDF = 1, VFO_AMNFE = 2, VFO_AMNFG = 3, VFO_EVMF = 4, VFO_EVBDF = 5 };
/* approximation codes */
enum { VFO_EXACT = 0, VFO_POLY = 1, VFO_RATIONAL = 2 };

#define VFO_MAXN 225 /* 15 x 15 */
#define VFO_MAXC 16

/* One approximant: p(z) (polynomial) or p(z)/q(z) (rational), coefficients in
 * increasing powers of z, as in the paper's tables (a_0 .. a_p). */
typedef struct {
  int num_len;
  int den_len; /* 0 for a polynomial */
  double num[VFO_MAXC];
  double den[VFO_MAXC];
} vfo_approximant;

typedef struct {
  int window;    /* odd w, n = w*w */
  int criterion; /* VFO_* */
  int approx;    /* VFO_EXACT / VFO_POLY / VFO_RATIONAL */
  double kappa;  /* AMNF kernel-width exponent, 0.33 in the paper */
  double exp_cutoff; /* AMNF: E(z) = 0 for z > exp_cutoff */
  double ent_cutoff; /* EVMF: ENT(z) = 0 for z < ent_cutoff */
  vfo_approximant acos_lo; /* BVDF: arccos(z) on [0, 0.5]          (Table 1) */
  vfo_approximant acos_hi; /* BVDF: 2 arcsin(tau/sqrt2) on [0,1/sqrt2] (Table 1) */
  vfo_approximant expo;    /* AMNF: exp(-z) on [0, exp_cutoff]        (Table 2) */
  vfo_approximant ent;     /* EVMF: z ln z on [ent_cutoff, 1]         (ENT table) */
} vfo_params;

/* Horner evaluation of sum_k c_k z^k. */
static double vfo_poly(const double* c, int len, double z) {
  double acc = 0.0;
  for (int k = len - 1; k >= 0; --k) acc = acc * z + c[k];
  return acc;
}

/* Sec. 2: evaluate a minimax polynomial or rational approximant. */
double vfo_eval_approximant(const vfo_approximant* a, double z) {
  double p = vfo_poly(a->num, a->num_len, z);
  if (a->den_len == 0) return p;
  return p / vfo_poly(a->den, a->den_len, z);
}

/* ---- pairwise and per-sample criteria (Sec. 3.1 - 3.3) ------------------ */

static double vfo_l2(const double* a, const double* b) {
  double s = 0.0;
  for (int k = 0; k < 3; ++k) s += (a[k] - b[k]) * (a[k] - b[k]);
  return sqrt(s);
}

static double vfo_l1(const double* a, const double* b) {
  double s = 0.0;
  for (int k = 0; k < 3; ++k) s += fabs(a[k] - b[k]);
  return s;
}

/* Sec. 3.1, BVDF equation, exact angle.  arccos of the normalised dot product
 * is evaluated as atan2(|a x b|, a.b), which is the same angle but keeps full
 * precision near 0, where arccos(z) of a rounded z loses half the bits. */
double vfo_angle_exact(const double* a, const double* b) {
  double na = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  double nb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  if (na == 0.0 || nb == 0.0) return acos(0.0);
  double cx = a[1] * b[2] - a[2] * b[1];
  double cy = a[2] * b[0] - a[0] * b[2];
  double cz = a[0] * b[1] - a[1] * b[0];
  double dot = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
  return atan2(sqrt(cx * cx + cy * cy + cz * cz), dot);
}

/* The literal form of the BVDF equation, arccos(dot / (|a| |b|)), kept for a
 * cross-check of vfo_angle_exact in the tests. */
double vfo_angle_acos(const double* a, const double* b) {
  double na = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  double nb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
  if (na == 0.0 || nb == 0.0) return acos(0.0);
  double z = (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (na * nb);
  if (z > 1.0) z = 1.0;
  if (z < -1.0) z = -1.0;
  return acos(z);
}

/* Sec. 3.1, the approximate angle: z in [0,1] (RGB vectors are
 * non-negative); for z < 0.5 the arccos approximant (ARCCOS row of Table 1);
 * for z >= 0.5 tau = sqrt(1 - z) and the approximant of 2 arcsin(tau/sqrt 2)
 * (ARCSIN row of Table 1), which equals arccos(z). */
double vfo_angle_approx(const vfo_params* p, const double* a, const double* b) {
  double na = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  double nb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
  double z = 0.0;
  if (na != 0.0 && nb != 0.0) z = (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (na * nb);
  if (z < 0.0) z = 0.0;
  if (z > 1.0) z = 1.0;
  if (z < 0.5) return vfo_eval_approximant(&p->acos_lo, z);
  double tau = sqrt(1.0 - z);
  return vfo_eval_approximant(&p->acos_hi, tau);
}

/* Sec. 3.2: the EXP function exp(-z) with the cut-off: 0 for arguments
 * outside [0, T]; inside, exact or through the approximant.  The cut-off is
 * read as part of the function the filter uses, for both variants (a cut-off
 * of +inf gives the plain exponential). */
double vfo_expneg(const vfo_params* p, double z) {
  if (z < 0.0 || z > p->exp_cutoff) return 0.0;
  if (p->approx == VFO_EXACT) return exp(-z);
  return vfo_eval_approximant(&p->expo, z);
}

/* Sec. 3.3: the ENT function z log z (natural log) with the cut-off: 0 for
 * arguments below T; above it, exact or through the approximant.  As for EXP
 * the cut-off belongs to both variants; a cut-off of 0 gives the plain
 * z log z with 0 log 0 = 0. */
double vfo_ent(const vfo_params* p, double z) {
  if (z < p->ent_cutoff || z <= 0.0) return 0.0;
  if (p->approx == VFO_EXACT) return z * log(z);
  return vfo_eval_approximant(&p->ent, z);
}

/* ---- one window ---------------------------------------------------------- */

/* Per-pixel diagnostics written next to the output (all optional). */
typedef struct {
  int32_t* sel;  /* selected raster index (0-based), -1 for a weighted mean */
  double* gap;   /* relative gap between the best aggregate and the best
                    aggregate of a sample whose vector differs (selection
                    filters), distance of the AMNF output to the nearest
                    rounding boundary, or |P_C - beta_C| / max for the EVMF
                    switch; each lowered to the relative distance of an
                    argument of E (AMNF) or of a P_j (EVMF switch) from its
                    cut-off where that is smaller; +inf when no competitor
                    exists */
  uint8_t* sw;   /* EVMF: 1 if the noise filtering branch was taken */
  double* yreal; /* AMNF: unrounded output, 3 per pixel */
} vfo_diag;

/* Sec. 3 / Fig. fig_window: gather the n window samples of (r,c) in raster
 * order, with the borders replicating the nearest pixel; off[i] (optional) is
 * the pixel index sample i was read from. */
static void vfo_gather(const uint8_t* img, int H, int W, int C, int w, int r, int c,
                       double x[][3], size_t* off) {
  int R = w / 2, i = 0;
  for (int dy = -R; dy <= R; ++dy) {
    int rr = r + dy;
    if (rr < 0) rr = 0;
    if (rr > H - 1) rr = H - 1;
    for (int dx = -R; dx <= R; ++dx) {
      int cc = c + dx;
      if (cc < 0) cc = 0;
      if (cc > W - 1) cc = W - 1;
      const uint8_t* px = img + ((size_t)rr * W + cc) * C;
      if (off) off[i] = (size_t)rr * W + cc;
      x[i][0] = px[0];
      x[i][1] = px[1];
      x[i][2] = px[2];
      ++i;
    }
  }
}

static int vfo_same(const double* a, const double* b) {
  return a[0] == b[0] && a[1] == b[1] && a[2] == b[2];
}

/* argmin_i agg[i], lowest index on an exact tie, plus the relative gap to the
 * best aggregate of a sample whose vector differs from the selected one. */
static int vfo_argmin(int n, const double* agg, double x[][3], double* gap) {
  int best = 0;
  for (int i = 1; i < n; ++i)
    if (agg[i] < agg[best]) best = i;
  double second = INFINITY;
  for (int i = 0; i < n; ++i)
    if (!vfo_same(x[i], x[best]) && agg[i] < second) second = agg[i];
  if (gap) *gap = isinf(second) ? INFINITY : (second - agg[best]) / agg[best];
  return best;
}

/* Sec. 3.3, first branch of Eq. (equ_evf) (the vector median filter):
 * aggregate of Euclidean distances, argmin. */
static int vfo_vmf_select(int n, double x[][3], double* gap) {
  double agg[VFO_MAXN];
  for (int i = 0; i < n; ++i) {
    agg[i] = 0.0;
    for (int j = 0; j < n; ++j)
      if (j != i) agg[i] += vfo_l2(x[i], x[j]);
  }
  return vfo_argmin(n, agg, x, gap);
}

/* Sec. 3.1, BVDF equation: aggregate of angles, argmin. */
static int vfo_bvdf_select(const vfo_params* p, int n, double x[][3], double* gap) {
  double agg[VFO_MAXN];
  for (int i = 0; i < n; ++i) {
    agg[i] = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      agg[i] += p->approx == VFO_EXACT ? vfo_angle_exact(x[i], x[j])
                                       : vfo_angle_approx(p, x[i], x[j]);
    }
  }
  return vfo_argmin(n, agg, x, gap);
}

/* Relative distance of z from the cut-off t (t > 0): the cut-off is a
 * threshold decision inside E and ENT (Sec. 3.2, 3.3), and a z this close to
 * it may fall on either side once rounded, like a near tie of the argmin. */
static double vfo_cut_gap(double z, double t) {
  return t > 0.0 ? fabs(z - t) / t : INFINITY;
}

/* Sec. 3.2, Eq. (equ_amnf): kernel-weighted mean of the window.  *cgap
 * (optional): the smallest vfo_cut_gap of the arguments z of E. */
static void vfo_amnf(const vfo_params* p, int n, double x[][3], double y[3], double* cgap) {
  int C = (n + 1) / 2 - 1; /* 0-based centre */
  double h[VFO_MAXN];
  double scale = pow((double)n, -p->kappa / 3.0);
  int all_zero = 1;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += vfo_l1(x[i], x[j]);
    h[i] = scale * s;
    if (h[i] != 0.0) all_zero = 0;
  }
  if (cgap) *cgap = INFINITY;
  if (all_zero) { /* constant window: every sample equals the centre */
    for (int k = 0; k < 3; ++k) y[k] = x[C][k];
    return;
  }
  double wsum = 0.0, acc[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < n; ++i) {
    double u;
    if (p->criterion == VFO_AMNFE) {
      u = vfo_l1(x[C], x[i]) / h[i]; /* ||(x_C - x_i)/h_i||_1 */
    } else {
      double d = vfo_l2(x[C], x[i]) / h[i];
      u = 0.5 * d * d; /* 0.5 ||(x_C - x_i)/h_i||_2^2 */
    }
    if (cgap) *cgap = fmin(*cgap, vfo_cut_gap(u, p->exp_cutoff));
    double wi = pow(h[i], -3.0) * vfo_expneg(p, u);
    wsum += wi;
    for (int k = 0; k < 3; ++k) acc[k] += wi * x[i][k];
  }
  for (int k = 0; k < 3; ++k) y[k] = acc[k] / wsum;
}

/* Sec. 3.3, Eq. (equ_evf): the entropy switch.  Returns 1 when the noise
 * filtering branch (P_C > beta_C) is taken. */
static int vfo_evmf_switch(const vfo_params* p, int n, double x[][3], double* gap) {
  int C = (n + 1) / 2 - 1;
  double mean[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) mean[k] += x[i][k];
  for (int k = 0; k < 3; ++k) mean[k] /= n;
  double r[VFO_MAXN], rsum = 0.0;
  for (int i = 0; i < n; ++i) {
    r[i] = vfo_l2(x[i], mean);
    rsum += r[i];
  }
  if (gap) *gap = INFINITY;
  if (rsum == 0.0) return 0; /* constant window: identity */
  double esum = 0.0, cgap = INFINITY;
  for (int j = 0; j < n; ++j) {
    esum += vfo_ent(p, r[j] / rsum);
    cgap = fmin(cgap, vfo_cut_gap(r[j] / rsum, p->ent_cutoff));
  }
  if (gap) *gap = cgap;
  if (esum == 0.0) return 0; /* no entropy left after the cut-off: identity */
  double PC = r[C] / rsum;
  double beta = vfo_ent(p, PC) / esum;
  if (gap) {
    double m = fmax(fabs(PC), fabs(beta));
    *gap = fmin(cgap, m > 0.0 ? fabs(PC - beta) / m : INFINITY);
  }
  return PC > beta;
}

static double vfo_round_gap(double v) {
  double f = v - floor(v);
  return fabs(f - 0.5);
}

static uint8_t vfo_round_u8(double v) {
  double q = nearbyint(v); /* round half to even (default rounding mode) */
  if (q < 0.0) q = 0.0;
  if (q > 255.0) q = 255.0;
  return (uint8_t)q;
}

/* Filter rows [row0, row1) of an H x W image with C interleaved channels
 * (C = 3 or 4; only the first three are colour) into `out` (same layout).
 * Returns 0, or -1 on a bad argument. */
int vfo_filter_rows(const uint8_t* img, int H, int W, int C, const vfo_params* p,
                    uint8_t* out, vfo_diag* dg, int row0, int row1) {
  int w = p->window;
  if (w < 1 || (w & 1) == 0 || w * w > VFO_MAXN || C < 3 || H < 1 || W < 1) return -1;
  int n = w * w, Cc = (n + 1) / 2 - 1;
  double (*x)[3] = malloc(sizeof(double[3]) * (size_t)n);
  size_t* off = malloc(sizeof(size_t) * (size_t)n);
  if (!x || !off) {
    free(x);
    free(off);
    return -1;
  }
  for (int r = row0; r < row1; ++r) {
    for (int c = 0; c < W; ++c) {
      size_t pix = (size_t)r * W + c;
      vfo_gather(img, H, W, C, w, r, c, x, off);
      double y[3];
      int sel = -1, sw = 0;
      double gap = INFINITY;
      switch (p->criterion) {
        case VFO_VMF:
          sel = vfo_vmf_select(n, x, &gap);
          break;
        case VFO_BVDF:
          sel = vfo_bvdf_select(p, n, x, &gap);
          break;
        case VFO_AMNFE:
        case VFO_AMNFG:
          double cgap;
          vfo_amnf(p, n, x, y, &cgap);
          gap = fmin(fmin(vfo_round_gap(y[0]), vfo_round_gap(y[1])), vfo_round_gap(y[2]));
          gap = fmin(gap, cgap);
          if (dg && dg->yreal)
            for (int k = 0; k < 3; ++k) dg->yreal[pix * 3 + k] = y[k];
          break;
        case VFO_EVMF:
        case VFO_EVBDF: {
          /* EVBDF: the generalised entropy vector filter of Sec. 3.3 (the
           * Euclidean distance of the filtering branch replaced by the angle
           * of Sec. 3.1); the switch is EVMF's */
          double sgap;
          sw = vfo_evmf_switch(p, n, x, &sgap);
          if (sw) {
            sel = p->criterion == VFO_EVMF ? vfo_vmf_select(n, x, &gap)
                                           : vfo_bvdf_select(p, n, x, &gap);
            gap = fmin(gap, sgap);
          } else {
            sel = Cc;
            gap = sgap;
          }
          break;
        }
        default:
          free(x);
          free(off);
          return -1;
      }
      /* bytes past the colour (RGBX): those of the selected sample's pixel
       * for a selection, of the centre pixel for a weighted mean */
      uint8_t* o = out + pix * C;
      if (sel >= 0) {
        for (int k = 0; k < 3; ++k) o[k] = (uint8_t)x[sel][k];
        for (int k = 3; k < C; ++k) o[k] = img[off[sel] * C + k];
      } else {
        for (int k = 0; k < 3; ++k) o[k] = vfo_round_u8(y[k]);
        for (int k = 3; k < C; ++k) o[k] = img[pix * C + k];
      }
      if (dg && dg->sel) dg->sel[pix] = sel;
      if (dg && dg->gap) dg->gap[pix] = gap;
      if (dg && dg->sw) dg->sw[pix] = (uint8_t)sw;
    }
  }
  free(x);
  free(off);
  return 0;
}

/* Whole image, rows split across `nthreads` OpenMP threads (each row is
 * independent; the result does not depend on the split). */
int vfo_filter(const uint8_t* img, int H, int W, int C, const vfo_params* p, uint8_t* out,
               vfo_diag* dg, int nthreads) {
  int err = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) reduction(| : err)
#endif
  for (int r = 0; r < H; ++r) err |= vfo_filter_rows(img, H, W, C, p, out, dg, r, r + 1) != 0;
  (void)nthreads;
  return err ? -1 : 0;
}

/* Per-window aggregates, exposed for the tests (permutation invariance, brute
 * force): window samples x[n][3] as given, returns agg[n] for the selection
 * criteria (VMF, BVDF). */
int vfo_window_aggregates(const vfo_params* p, int n, const double* xs, double* agg) {
  if (n < 1 || n > VFO_MAXN) return -1;
  double (*x)[3] = (double (*)[3])xs;
  for (int i = 0; i < n; ++i) {
    agg[i] = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      if (p->criterion == VFO_BVDF)
        agg[i] += p->approx == VFO_EXACT ? vfo_angle_exact(x[i], x[j])
                                         : vfo_angle_approx(p, x[i], x[j]);
      else
        agg[i] += vfo_l2(x[i], x[j]);
    }
  }
  return 0;
}

/* EVMF switch of one window given as x[n][3], exposed for the tests. */
int vfo_window_evmf_switch(const vfo_params* p, int n, const double* xs, double* gap) {
  return vfo_evmf_switch(p, n, (double (*)[3])xs, gap);
}

/* AMNF output of one window given as x[n][3], exposed for the tests. */
int vfo_window_amnf(const vfo_params* p, int n, const double* xs, double* y) {
  vfo_amnf(p, n, (double (*)[3])xs, y, NULL);
  return 0;
}
