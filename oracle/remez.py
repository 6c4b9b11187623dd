"""Minimax polynomial fit by the Remez exchange algorithm (Sec. 2), FP64.

TEST INFRASTRUCTURE ONLY: part of the oracle.  The product library carries its
own, independently written fit; nothing here is imported by it.

Sec. 2 defines the target: among polynomials P of degree <= p, minimise
eps = max_{z in [a,b]} |f(z) - P(z)|.  The paper computes it with the Remez
exchange algorithm, "an iterative method that uses Lagrangian interpolation".
The steps below follow that description:

1. start from a reference of p+2 points (the Chebyshev extrema of [a,b]);
2. on the reference, find the levelled error E and the polynomial P with
   f(x_k) - P(x_k) = (-1)^k E.  With the barycentric (Lagrange) weights
   lam_k = 1 / prod_{m != k} (x_k - x_m) of the p+2 points, the (p+1)-th divided
   difference of f - P vanishes for any P of degree <= p, which gives
   E = sum_k lam_k f(x_k) / sum_k lam_k (-1)^k, and P is the Lagrange
   interpolant of the values f(x_k) - (-1)^k E;
3. locate the extrema of the error f - P on [a,b] and exchange the reference
   for p+2 alternating extrema containing the largest one;
4. repeat until the extrema are level (max |e| / min |e(x_k)| - 1 < tol;
   1e-8 is the level that FP64 evaluation of the error can resolve).

The monomial coefficients (a_0 .. a_p, as in Tables 1 and 2) are obtained by
expanding the Lagrange interpolant of step 2.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import polynomial as npoly


def _bary_weights(x: np.ndarray) -> np.ndarray:
    lam = np.empty_like(x)
    for k in range(len(x)):
        d = x[k] - np.delete(x, k)
        lam[k] = 1.0 / np.prod(d)
    return lam


def _lagrange_monomial(xs: np.ndarray, ys: np.ndarray, a: float, b: float) -> np.ndarray:
    """Monomial coefficients (increasing powers of z) of the Lagrange
    interpolant.  The Lagrange basis is expanded in t = (z - c) / h, c and h
    the centre and half-width of [a, b], where it is well conditioned, and
    then rewritten in powers of z."""
    c, h = 0.5 * (a + b), 0.5 * (b - a)
    ts = (xs - c) / h
    coef_t = np.zeros(len(xs))
    for k in range(len(xs)):
        others = np.delete(ts, k)
        basis = npoly.polyfromroots(others) / np.prod(ts[k] - others)
        coef_t = coef_t + ys[k] * basis
    # sum_k coef_t[k] ((z - c) / h)^k
    coef = np.zeros(len(xs))
    lin = np.array([-c / h, 1.0 / h])
    power = np.array([1.0])
    for k in range(len(xs)):
        coef[: len(power)] += coef_t[k] * power
        power = npoly.polymul(power, lin)
    return coef


def _lagrange_eval(xs: np.ndarray, ys: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Second barycentric form of the Lagrange interpolant, evaluated at z."""
    lam = _bary_weights(xs)
    z = np.asarray(z, dtype=np.float64)
    diff = z[:, None] - xs[None, :]
    exact = diff == 0.0
    diff[exact] = 1.0
    t = lam[None, :] / diff
    val = (t @ ys) / t.sum(axis=1)
    hit = exact.any(axis=1)
    if hit.any():
        val[hit] = ys[np.argmax(exact[hit], axis=1)]
    return val


def _golden_max(g, lo: float, hi: float, iters: int = 80) -> float:
    """Maximise a unimodal function g on [lo, hi] by golden-section search."""
    r = (np.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c, d = b - r * (b - a), a + r * (b - a)
    gc, gd = g(c), g(d)
    for _ in range(iters):
        if gc > gd:
            b, d, gd = d, c, gc
            c = b - r * (b - a)
            gc = g(c)
        else:
            a, c, gc = c, d, gd
            d = a + r * (b - a)
            gd = g(d)
    return 0.5 * (a + b)


class MinimaxFit:
    """Result of a fit: coefficients a_0..a_p, error eps, final reference."""

    def __init__(self, coef, eps, levelled, reference, a, b, iterations):
        self.coef = np.asarray(coef, dtype=np.float64)
        self.eps = float(eps)
        self.levelled = float(levelled)
        self.reference = np.asarray(reference, dtype=np.float64)
        self.a, self.b = float(a), float(b)
        self.iterations = iterations

    def __call__(self, z):
        return npoly.polyval(np.asarray(z, dtype=np.float64), self.coef)


def remez(f, a: float, b: float, degree: int, grid: int = 20001, tol: float = 1e-8,
          max_iter: int = 60) -> MinimaxFit:
    """Degree-`degree` minimax polynomial of f on [a, b] (Sec. 2)."""
    p = degree
    k = np.arange(p + 2)
    # step 1: Chebyshev extrema of [a, b]
    x = 0.5 * (a + b) - 0.5 * (b - a) * np.cos(np.pi * k / (p + 1))
    sgn = (-1.0) ** k
    zs = np.linspace(a, b, grid)
    fz = f(zs)
    E = 0.0
    for it in range(1, max_iter + 1):
        # step 2: levelled error and Lagrange interpolant
        fx = f(x)
        lam = _bary_weights(x)
        E = float(np.dot(lam, fx) / np.dot(lam, sgn))
        nodes, vals = x[: p + 1], fx[: p + 1] - sgn[: p + 1] * E

        def err(z, nodes=nodes, vals=vals):
            z = np.atleast_1d(np.asarray(z, dtype=np.float64))
            return f(z) - _lagrange_eval(nodes, vals, z)

        # step 3: extrema of the error, refined by golden-section search
        e = fz - _lagrange_eval(nodes, vals, zs)
        de = np.diff(e)
        turn = np.nonzero((de[:-1] * de[1:] <= 0.0) & (e[1:-1] != 0.0))[0] + 1
        cand = [0] + [int(i) for i in turn] + [grid - 1]
        pts, vals_e = [], []
        for i in cand:
            if i in (0, grid - 1):
                xi = zs[i]
            else:
                s = np.sign(e[i])
                xi = _golden_max(lambda t, s=s: s * float(err(t)[0]), zs[i - 1], zs[i + 1])
            ei = float(err(xi)[0])
            # keep one point per run of equal sign: the largest
            if pts and np.sign(ei) == np.sign(vals_e[-1]):
                if abs(ei) > abs(vals_e[-1]):
                    pts[-1], vals_e[-1] = xi, ei
            else:
                pts.append(xi)
                vals_e.append(ei)
        # reduce to p+2 alternating points containing the global maximum
        while len(pts) > p + 2:
            if abs(vals_e[0]) < abs(vals_e[-1]):
                pts.pop(0)
                vals_e.pop(0)
            else:
                pts.pop()
                vals_e.pop()
        emax = max(abs(v) for v in vals_e)
        emin = min(abs(v) for v in vals_e)
        if len(pts) == p + 2:
            x = np.array(pts)
            sgn = np.sign(np.array(vals_e))
        # step 4: stop when the error is levelled
        if emin > 0.0 and emax / emin - 1.0 < tol:
            break
    coef = _lagrange_monomial(nodes, vals, a, b)
    # eps: maximum error of the final polynomial on the interval
    e_final = np.abs(fz - npoly.polyval(zs, coef))
    eps = max(float(e_final.max()), emax)
    return MinimaxFit(coef, eps, abs(E), x, a, b, it)


def max_error(f, approx, a: float, b: float, samples: int = 2_000_001) -> float:
    """max_{z in [a,b]} |f(z) - approx(z)| on a dense uniform grid."""
    z = np.linspace(a, b, samples)
    return float(np.max(np.abs(f(z) - approx(z))))


def equioscillation(f, fit: MinimaxFit):
    """Signed error at the final reference points (p+2 of them)."""
    return f(fit.reference) - fit(fit.reference)


# ---------------------------------------------------------------- rationals

class RationalFit:
    """Minimax rational p/q: numerator a_0..a_m, denominator b_0..b_n (b_0 = 1),
    error eps, final reference of m+n+2 points."""

    def __init__(self, num, den, eps, levelled, reference, a, b, iterations):
        self.num = np.asarray(num, dtype=np.float64)
        self.den = np.asarray(den, dtype=np.float64)
        self.eps = float(eps)
        self.levelled = float(levelled)
        self.reference = np.asarray(reference, dtype=np.float64)
        self.a, self.b = float(a), float(b)
        self.iterations = iterations

    def __call__(self, z):
        z = np.asarray(z, dtype=np.float64)
        return npoly.polyval(z, self.num) / npoly.polyval(z, self.den)


def rational_remez(f, a: float, b: float, m: int, n: int, grid: int = 20001,
                   tol: float = 1e-7, max_iter: int = 80) -> RationalFit:
    """Best rational approximation p/q, deg p <= m, deg q <= n, of f on [a, b]
    in the maximum norm (Sec. 2, the class R^n_m and its existence theorem).

    A non-degenerate best approximation is characterised by an error that
    equioscillates on m+n+2 points, so the same exchange as for polynomials
    applies, with step 2 replaced: on the reference x_k the conditions
    f(x_k) - p(x_k)/q(x_k) = (-1)^k E read p(x_k) - f(x_k) q(x_k) =
    -(-1)^k E q(x_k), linear in the coefficients of p and q for a given E.
    All m+n+2 of them (coefficients of p and q, q unnormalised) form the
    generalised eigenproblem A c = E B c; the level E is the eigenvalue of
    smallest magnitude whose q keeps one sign on [a, b] (no pole).  p and q
    are carried in the Chebyshev basis of [a, b] for conditioning and
    expanded to monomials at the end, with q(0) scaled to 1.  The exchange
    stops when the extrema are level to 1e-7 (the quotient's FP64 rounding
    resolves no finer).
    """
    from numpy.polynomial import chebyshev as C
    from scipy.linalg import eig

    N = m + n + 2
    mid, half = 0.5 * (a + b), 0.5 * (b - a)
    k = np.arange(N)
    t = -np.cos(np.pi * k / (N - 1))   # reference in [-1, 1] (Chebyshev extrema)
    ts = np.linspace(-1.0, 1.0, grid)
    zs = mid + half * ts
    fz = f(zs)
    sgn = (-1.0) ** k

    def solve(t):
        fx = f(mid + half * t)
        Tp = C.chebvander(t, m)                 # N x (m+1)
        Tq = C.chebvander(t, n)                 # N x (n+1)
        A = np.hstack([Tp, -fx[:, None] * Tq])
        B = np.hstack([np.zeros_like(Tp), -(sgn[:, None] * Tq)])
        w, V = eig(A, B)
        best = None
        for lam, v in zip(w, V.T):
            if not np.isfinite(lam) or abs(lam.imag) > 1e-9 * max(1.0, abs(lam.real)):
                continue
            v = np.real(v)
            q = C.chebval(ts, v[m + 1:])
            if not (np.all(q > 0.0) or np.all(q < 0.0)):
                continue
            if best is None or abs(lam.real) < abs(best[0]):
                best = (lam.real, v)
        if best is None:
            raise RuntimeError("no pole-free rational on the reference")
        E, v = best
        return E, v[: m + 1], v[m + 1:]

    def err_of(pc, qc):
        def err(tt):
            tt = np.atleast_1d(np.asarray(tt, dtype=np.float64))
            return f(mid + half * tt) - C.chebval(tt, pc) / C.chebval(tt, qc)
        return err

    E, pc, qc = 0.0, None, None
    emax = np.inf
    for it in range(1, max_iter + 1):
        E, pc, qc = solve(t)
        err = err_of(pc, qc)
        e = fz - C.chebval(ts, pc) / C.chebval(ts, qc)
        de = np.diff(e)
        turn = np.nonzero((de[:-1] * de[1:] <= 0.0) & (e[1:-1] != 0.0))[0] + 1
        cand = [0] + [int(i) for i in turn] + [grid - 1]
        pts, vals_e = [], []
        for i in cand:
            if i in (0, grid - 1):
                xi = ts[i]
            else:
                s = np.sign(e[i])
                xi = _golden_max(lambda u, s=s: s * float(err(u)[0]), ts[i - 1], ts[i + 1])
            ei = float(err(xi)[0])
            if pts and np.sign(ei) == np.sign(vals_e[-1]):
                if abs(ei) > abs(vals_e[-1]):
                    pts[-1], vals_e[-1] = xi, ei
            else:
                pts.append(xi)
                vals_e.append(ei)
        while len(pts) > N:
            if abs(vals_e[0]) < abs(vals_e[-1]):
                pts.pop(0)
                vals_e.pop(0)
            else:
                pts.pop()
                vals_e.pop()
        emax = max(abs(v) for v in vals_e)
        emin = min(abs(v) for v in vals_e)
        if len(pts) == N:
            t = np.array(pts)
            sgn = np.sign(np.array(vals_e))
        if emin > 0.0 and emax / emin - 1.0 < tol:
            break
        if emax <= 1e-13 * float(np.max(np.abs(fz))):
            break  # at the FP64 rounding level of the quotient: nothing to level
    # monomial coefficients in z: substitute t = (z - mid) / half
    pm = _cheb_to_monomial(pc, mid, half)
    qm = _cheb_to_monomial(qc, mid, half)
    pm, qm = pm / qm[0], qm / qm[0]
    e_final = np.abs(fz - npoly.polyval(zs, pm) / npoly.polyval(zs, qm))
    eps = max(float(e_final.max()), emax)
    return RationalFit(pm, qm, eps, abs(E), mid + half * t, a, b, it)


def _cheb_to_monomial(c, mid: float, half: float) -> np.ndarray:
    """Monomial coefficients in z of sum_j c_j T_j((z - mid) / half)."""
    from numpy.polynomial import chebyshev as C
    pt = C.cheb2poly(c)                      # coefficients in t
    out = np.zeros(len(pt))
    lin = np.array([-mid / half, 1.0 / half])  # t as a polynomial in z
    powt = np.array([1.0])
    for j, cj in enumerate(pt):
        out[: len(powt)] += cj * powt
        powt = npoly.polymul(powt, lin)
    return out
