// vf_remez.cpp -- the library's host-side minimax fit (Sec. 2), FP64.
//
// Remez exchange for the best polynomial approximation of degree p in the
// Chebyshev (maximum) norm.  Formulation used here: on a reference of p+2
// points t_k of [-1, 1] (the interval mapped affinely), solve the linear
// system  sum_m c_m T_m(t_k) + (-1)^k E = f(t_k)  for the Chebyshev
// coefficients c and the levelled error E; sample the error, take the
// extremum of every run of one sign (refined by ternary search) and keep p+2
// alternating ones containing the largest as the new reference; stop when
// the extrema are level.  The result is re-expanded in powers of
// the original argument (a_0 .. a_p, as the paper tabulates them).
#include <algorithm>
#include <cmath>
#include <vector>

#include "vf_internal.h"

namespace vf {
namespace {

double target(int fn, double x) {
  switch (fn) {
    case 0: return std::acos(x);                                // arccos(z)
    case 1: return 2.0 * std::asin(x / std::sqrt(2.0));         // 2 arcsin(tau/sqrt2)
    case 2: return std::exp(-x);                                // exp(-z)
    case 3: return x > 0.0 ? x * std::log(x) : 0.0;             // z ln z
    case 4: {  // 2 atan(sqrt s) / sqrt s: the exact angle's arctangent, A = u P(u^2)
      if (x <= 0.0) return 2.0;
      const double r = std::sqrt(x);
      return 2.0 * std::atan(r) / r;
    }
    default: return 0.0;
  }
}

// Chebyshev polynomials T_0..T_p at t.
void cheb(double t, int p, double* T) {
  T[0] = 1.0;
  if (p >= 1) T[1] = t;
  for (int m = 2; m <= p; ++m) T[m] = 2.0 * t * T[m - 1] - T[m - 2];
}

// Gaussian elimination with partial pivoting, n x n system in row-major A.
bool solve(std::vector<double>& A, std::vector<double>& b, int n) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[r * n + col]) > std::fabs(A[piv * n + col])) piv = r;
    if (A[piv * n + col] == 0.0) return false;
    if (piv != col) {
      for (int c = 0; c < n; ++c) std::swap(A[piv * n + c], A[col * n + c]);
      std::swap(b[piv], b[col]);
    }
    for (int r = col + 1; r < n; ++r) {
      double f = A[r * n + col] / A[col * n + col];
      for (int c = col; c < n; ++c) A[r * n + c] -= f * A[col * n + c];
      b[r] -= f * b[col];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int c = r + 1; c < n; ++c) s -= A[r * n + c] * b[c];
    b[r] = s / A[r * n + r];
  }
  return true;
}

struct Fit {
  int fn, p;
  double lo, hi;
  std::vector<double> c;  // Chebyshev coefficients in t
  double x_of(double t) const { return 0.5 * (lo + hi) + 0.5 * (hi - lo) * t; }
  double err(double t) const {
    double T[16];
    cheb(t, p, T);
    double s = 0.0;
    for (int m = 0; m <= p; ++m) s += c[m] * T[m];
    return target(fn, x_of(t)) - s;
  }
};

}  // namespace

bool remez_fit(int fn, int degree, double lo, double hi, double* coef, double* eps) {
  const int p = degree, n = p + 2;
  if (p < 1 || p > 12 || !(hi > lo)) return false;
  Fit F{fn, p, lo, hi, std::vector<double>(p + 1, 0.0)};
  std::vector<double> ref(n);
  for (int k = 0; k < n; ++k) ref[k] = -std::cos(M_PI * k / (p + 1));

  const int G = 4097;
  double level = 0.0;
  for (int it = 0; it < 40; ++it) {
    std::vector<double> A(n * n), b(n);
    for (int k = 0; k < n; ++k) {
      double T[16];
      cheb(ref[k], p, T);
      for (int m = 0; m <= p; ++m) A[k * n + m] = T[m];
      A[k * n + p + 1] = (k & 1) ? -1.0 : 1.0;
      b[k] = target(fn, F.x_of(ref[k]));
    }
    if (!solve(A, b, n)) return false;
    for (int m = 0; m <= p; ++m) F.c[m] = b[m];
    level = std::fabs(b[p + 1]);

    // sample the error; collect the extremum of every run of one sign
    std::vector<double> ts, es;
    double run_t = -1.0, run_e = F.err(-1.0);
    for (int g = 1; g < G; ++g) {
      double t = -1.0 + 2.0 * g / (G - 1);
      double e = F.err(t);
      if ((e > 0) == (run_e > 0)) {
        if (std::fabs(e) > std::fabs(run_e)) run_t = t, run_e = e;
      } else {
        ts.push_back(run_t);
        es.push_back(run_e);
        run_t = t;
        run_e = e;
      }
    }
    ts.push_back(run_t);
    es.push_back(run_e);
    // refine interior extrema by ternary search on |e| within one sample step
    const double h = 2.0 / (G - 1);
    for (size_t k = 0; k < ts.size(); ++k) {
      if (ts[k] <= -1.0 || ts[k] >= 1.0) continue;
      double a = std::max(-1.0, ts[k] - h), c = std::min(1.0, ts[k] + h);
      double sg = es[k] > 0 ? 1.0 : -1.0;
      for (int r = 0; r < 100; ++r) {
        double m1 = a + (c - a) / 3.0, m2 = c - (c - a) / 3.0;
        if (sg * F.err(m1) < sg * F.err(m2)) a = m1; else c = m2;
      }
      ts[k] = 0.5 * (a + c);
      es[k] = F.err(ts[k]);
    }
    // keep n alternating extrema containing the largest
    while ((int)ts.size() > n) {
      if (std::fabs(es.front()) < std::fabs(es.back())) {
        ts.erase(ts.begin());
        es.erase(es.begin());
      } else {
        ts.pop_back();
        es.pop_back();
      }
    }
    if ((int)ts.size() < n) break;  // cannot happen for the library's targets
    double emax = 0.0, emin = 1e300;
    for (double e : es) emax = std::max(emax, std::fabs(e)), emin = std::min(emin, std::fabs(e));
    ref = ts;
    if (emax - emin <= 1e-9 * emax) break;
  }

  // re-expand sum_m c_m T_m((x - mid) / half) in powers of x
  const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
  std::vector<std::vector<double>> Tm(p + 1, std::vector<double>(p + 1, 0.0));  // T_m in t
  Tm[0][0] = 1.0;
  if (p >= 1) Tm[1][1] = 1.0;
  for (int m = 2; m <= p; ++m)
    for (int k = 0; k <= m; ++k)
      Tm[m][k] = (k > 0 ? 2.0 * Tm[m - 1][k - 1] : 0.0) - Tm[m - 2][k];
  std::vector<double> in_t(p + 1, 0.0);
  for (int m = 0; m <= p; ++m)
    for (int k = 0; k <= m; ++k) in_t[k] += F.c[m] * Tm[m][k];
  // t^k = ((x - mid) / half)^k, binomial expansion
  std::vector<double> out(p + 1, 0.0);
  for (int k = 0; k <= p; ++k) {
    double scale = in_t[k] / std::pow(half, k);
    double binom = 1.0;
    for (int j = 0; j <= k; ++j) {  // C(k, j) x^j (-mid)^(k-j)
      out[j] += scale * binom * std::pow(-mid, k - j);
      binom = binom * (k - j) / (j + 1);
    }
  }
  for (int k = 0; k <= p; ++k) coef[k] = out[k];
  // eps: maximum error of the monomial form on a dense grid
  double e = 0.0;
  for (int g = 0; g <= 20000; ++g) {
    double x = lo + (hi - lo) * g / 20000.0, s = 0.0;
    for (int k = p; k >= 0; --k) s = s * x + coef[k];
    e = std::max(e, std::fabs(target(fn, x) - s));
  }
  *eps = std::max(e, level);
  return true;
}

// ---------------------------------------------------------------- rationals
//
// Best rational approximation p/q, deg p <= m, deg q <= n, of f in the
// maximum norm (Sec. 2, the class R^n_m).  A non-degenerate best
// approximation has an error that equioscillates on m+n+2 points, so the
// exchange above carries over; only the solve on the reference changes.  On
// the reference t_k the conditions f - p/q = (-1)^k E, i.e.
//   p(t_k) - f(t_k) q(t_k) + (-1)^k E q(t_k) = 0,
// are bilinear in (q, E).  They are solved by fixed-point iteration: with
// q(t_k) in the E term taken from the previous iterate, the system is linear
// in the Chebyshev coefficients of p (m+1), of q with its T_0 coefficient
// fixed to 1 (n), and E; it is re-solved until E settles (a few rounds).
// Starting from q = 1 this is the polynomial solve.
namespace {

struct RFit {
  int fn, m, n;
  double lo, hi;
  std::vector<double> p, q;  // Chebyshev coefficients in t; q[0] = 1
  double x_of(double t) const { return 0.5 * (lo + hi) + 0.5 * (hi - lo) * t; }
  double qv(double t) const {
    double T[16];
    cheb(t, n, T);
    double s = 0.0;
    for (int j = 0; j <= n; ++j) s += q[j] * T[j];
    return s;
  }
  double err(double t) const {
    double T[16];
    cheb(t, m, T);
    double s = 0.0;
    for (int j = 0; j <= m; ++j) s += p[j] * T[j];
    return target(fn, x_of(t)) - s / qv(t);
  }
};

// Monomial coefficients in x of sum_j c_j T_j((x - mid) / half).
std::vector<double> to_monomial(const std::vector<double>& c, double mid, double half) {
  const int d = (int)c.size() - 1;
  std::vector<std::vector<double>> Tm(d + 1, std::vector<double>(d + 1, 0.0));
  Tm[0][0] = 1.0;
  if (d >= 1) Tm[1][1] = 1.0;
  for (int m = 2; m <= d; ++m)
    for (int k = 0; k <= m; ++k) Tm[m][k] = (k > 0 ? 2.0 * Tm[m - 1][k - 1] : 0.0) - Tm[m - 2][k];
  std::vector<double> in_t(d + 1, 0.0), out(d + 1, 0.0);
  for (int m = 0; m <= d; ++m)
    for (int k = 0; k <= m; ++k) in_t[k] += c[m] * Tm[m][k];
  for (int k = 0; k <= d; ++k) {
    const double scale = in_t[k] / std::pow(half, k);
    double binom = 1.0;
    for (int j = 0; j <= k; ++j) {
      out[j] += scale * binom * std::pow(-mid, k - j);
      binom = binom * (k - j) / (j + 1);
    }
  }
  return out;
}

}  // namespace

bool remez_rational_fit(int fn, int m, int n, double lo, double hi, double* num, double* den,
                        double* eps) {
  const int N = m + n + 2;
  if (m < 1 || n < 1 || m > 8 || n > 8 || !(hi > lo)) return false;
  RFit F{fn, m, n, lo, hi, std::vector<double>(m + 1, 0.0), std::vector<double>(n + 1, 0.0)};
  F.q[0] = 1.0;
  std::vector<double> ref(N);
  for (int k = 0; k < N; ++k) ref[k] = -std::cos(M_PI * k / (N - 1));
  std::vector<double> sg(N);
  for (int k = 0; k < N; ++k) sg[k] = (k & 1) ? -1.0 : 1.0;
  double fmax = 0.0;
  for (int g = 0; g <= 200; ++g) fmax = std::max(fmax, std::fabs(target(fn, F.x_of(-1.0 + g / 100.0))));

  const int G = 8193;
  double level = 0.0;
  for (int it = 0; it < 60; ++it) {
    // solve on the reference: fixed point in the E q(t_k) term
    std::vector<double> qprev(N);
    for (int k = 0; k < N; ++k) qprev[k] = F.qv(ref[k]);
    double E = 0.0;
    for (int s = 0; s < 50; ++s) {
      std::vector<double> A(N * N, 0.0), b(N);
      for (int k = 0; k < N; ++k) {
        double Tp[16], Tq[16];
        cheb(ref[k], m, Tp);
        cheb(ref[k], n, Tq);
        const double fk = target(fn, F.x_of(ref[k]));
        for (int j = 0; j <= m; ++j) A[k * N + j] = Tp[j];
        for (int j = 1; j <= n; ++j) A[k * N + m + j] = -fk * Tq[j];
        A[k * N + m + n + 1] = sg[k] * qprev[k];
        b[k] = fk;  // the fixed q_0 = 1 term moved to the right
      }
      if (!solve(A, b, N)) return false;
      for (int j = 0; j <= m; ++j) F.p[j] = b[j];
      for (int j = 1; j <= n; ++j) F.q[j] = b[m + j];
      const double Enew = b[m + n + 1];
      for (int k = 0; k < N; ++k) qprev[k] = F.qv(ref[k]);
      const bool settled = std::fabs(Enew - E) <= 1e-14 * std::fabs(Enew);
      E = Enew;
      if (settled) break;
    }
    level = std::fabs(E);
    // the denominator must keep its sign on [-1, 1] (no pole)
    for (int g = 0; g < G; ++g)
      if (!(F.qv(-1.0 + 2.0 * g / (G - 1)) > 0.0)) return false;

    // error extrema, one per run of one sign, refined by ternary search
    std::vector<double> ts, es;
    double run_t = -1.0, run_e = F.err(-1.0);
    for (int g = 1; g < G; ++g) {
      const double t = -1.0 + 2.0 * g / (G - 1), e = F.err(t);
      if ((e > 0) == (run_e > 0)) {
        if (std::fabs(e) > std::fabs(run_e)) run_t = t, run_e = e;
      } else {
        ts.push_back(run_t);
        es.push_back(run_e);
        run_t = t;
        run_e = e;
      }
    }
    ts.push_back(run_t);
    es.push_back(run_e);
    const double h = 2.0 / (G - 1);
    for (size_t k = 0; k < ts.size(); ++k) {
      if (ts[k] <= -1.0 || ts[k] >= 1.0) continue;
      double a = std::max(-1.0, ts[k] - h), c = std::min(1.0, ts[k] + h);
      const double s = es[k] > 0 ? 1.0 : -1.0;
      for (int r = 0; r < 100; ++r) {
        const double m1 = a + (c - a) / 3.0, m2 = c - (c - a) / 3.0;
        if (s * F.err(m1) < s * F.err(m2)) a = m1; else c = m2;
      }
      ts[k] = 0.5 * (a + c);
      es[k] = F.err(ts[k]);
    }
    while ((int)ts.size() > N) {
      if (std::fabs(es.front()) < std::fabs(es.back())) {
        ts.erase(ts.begin());
        es.erase(es.begin());
      } else {
        ts.pop_back();
        es.pop_back();
      }
    }
    if ((int)ts.size() < N) break;
    double emax = 0.0, emin = 1e300;
    for (double e : es) emax = std::max(emax, std::fabs(e)), emin = std::min(emin, std::fabs(e));
    ref = ts;
    for (int k = 0; k < N; ++k) sg[k] = es[k] > 0 ? 1.0 : -1.0;
    if (emax - emin <= 1e-7 * emax || emax <= 1e-13 * fmax) break;
  }

  const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
  std::vector<double> pm = to_monomial(F.p, mid, half), qm = to_monomial(F.q, mid, half);
  if (qm[0] == 0.0) return false;
  for (int j = 0; j <= m; ++j) num[j] = pm[j] / qm[0];
  for (int j = 0; j <= n; ++j) den[j] = qm[j] / qm[0];  // den[0] = 1 exactly
  double e = 0.0;
  for (int g = 0; g <= 20000; ++g) {
    const double x = lo + (hi - lo) * g / 20000.0;
    double pv = 0.0, qv = 0.0;
    for (int k = m; k >= 0; --k) pv = pv * x + num[k];
    for (int k = n; k >= 0; --k) qv = qv * x + den[k];
    e = std::max(e, std::fabs(target(fn, x) - pv / qv));
  }
  *eps = std::max(e, level);
  return true;
}

bool approximant_error(int fn, const double* num, int num_len, const double* den, int den_len,
                       double lo, double hi, double* eps) {
  double e = 0.0;
  int sign = 0;  // sign of the denominator at lo; it must keep it on [lo, hi]
  for (int g = 0; g <= 20000; ++g) {
    const double x = lo + (hi - lo) * g / 20000.0;
    double pv = 0.0, qv = 1.0;
    for (int k = num_len - 1; k >= 0; --k) pv = pv * x + num[k];
    if (den_len > 0) {
      qv = 0.0;
      for (int k = den_len - 1; k >= 0; --k) qv = qv * x + den[k];
      const int sg = qv > 0.0 ? 1 : (qv < 0.0 ? -1 : 0);
      if (sg == 0 || (sign != 0 && sg != sign)) return false;  // a pole on the interval
      sign = sg;
    }
    e = std::max(e, std::fabs(target(fn, x) - pv / qv));
  }
  *eps = e;
  return std::isfinite(e);
}

}  // namespace vf
