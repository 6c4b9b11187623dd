"""Pins of the oracle's Remez fit and approximants against what the paper
prints (Tables 1, 2, tab_exp_rat, tab_ent_rat) and against textbook closed
forms.  CPU only."""
import math

import numpy as np
import pytest

from oracle import approximants as AP
from oracle import paper_tables as PT
from oracle import remez as R


def _poly(c):
    return lambda z: np.polynomial.polynomial.polyval(np.asarray(z, dtype=np.float64), c)


def _rat(num, den):
    P = np.polynomial.polynomial
    return lambda z: P.polyval(np.asarray(z), num) / P.polyval(np.asarray(z), den)


def _sup_diff(p, q, a, b, n=200001):
    z = np.linspace(a, b, n)
    return float(np.max(np.abs(p(z) - q(z))))


def test_chebyshev_closed_form():
    """Textbook: the best degree-4 approximation of z^5 on [-1, 1] is
    z^5 - T_5(z)/16 = 1.25 z^3 - 0.3125 z, with error 2^-4."""
    fit = R.remez(lambda z: np.asarray(z) ** 5, -1.0, 1.0, 4)
    assert fit.eps == pytest.approx(1.0 / 16.0, rel=1e-9)
    np.testing.assert_allclose(fit.coef, [0.0, -0.3125, 0.0, 1.25, 0.0], atol=1e-9)


def test_linear_closed_form():
    """Textbook: the best line to a convex f on [a, b] has slope
    (f(b) - f(a)) / (b - a) and touches the error level at a, at the point
    where f' equals that slope, and at b.  For exp on [0, 1]: slope e - 1,
    tangent point ln(e - 1)."""
    fit = R.remez(np.exp, 0.0, 1.0, 1)
    m = math.e - 1.0
    xs = math.log(m)
    eps = 0.5 * (1.0 - (math.exp(xs) - m * xs))  # half the gap at a vs xs
    assert fit.coef[1] == pytest.approx(m, rel=1e-9)
    assert fit.eps == pytest.approx(abs(eps), rel=1e-8)


@pytest.mark.parametrize("row", ["table1_arcsin", "table1_arccos"])
def test_table1(golden, row):
    g = golden[row]
    name = "acos_hi" if row.endswith("arcsin") else "acos_lo"
    a, b = g["interval"]
    fit = AP.fit(name, 4, a, b)
    # the error of the fit is the printed eps (to the printed precision of a
    # slightly different Remez run)
    assert fit.eps == pytest.approx(g["eps"], rel=1e-4)
    # the fitted polynomial and the printed one are the same function up to a
    # small fraction of eps
    assert _sup_diff(fit, _poly(g["coef"]), a, b) < 0.02 * g["eps"]
    # coefficients agree to about the printed digits: the ARCCOS row's a_2
    # (-1.429899e-02) sits 1.3e-5 (relative) from the fit, whose a_2 has the
    # magnitude of the ARCSIN row's a_2; the printed eps of that row is 5e-5
    # above the fitted one, so the paper's run stopped slightly short of level
    np.testing.assert_allclose(fit.coef, g["coef"], rtol=2e-5, atol=2e-10)


@pytest.mark.parametrize("deg", ["2", "3", "4"])
def test_table2(golden, deg):
    g = golden["table2_exp"]
    a, b = g["interval"]
    row = g["rows"][deg]
    fit = AP.fit("exp", int(deg), a, b)
    assert fit.eps == pytest.approx(row["eps"], rel=1e-4)
    assert _sup_diff(fit, _poly(row["coef"]), a, b) < 0.001 * row["eps"]
    np.testing.assert_allclose(fit.coef, row["coef"], rtol=1e-5)


@pytest.mark.parametrize("name,interval", [
    ("acos_lo", AP.ACOS_LO_INTERVAL), ("acos_hi", AP.ACOS_HI_INTERVAL),
    ("exp", (0.0, 10.0)), ("ent", (0.05, 1.0)), ("exp", (0.0, 1.6)), ("ent", (0.018, 1.0))])
@pytest.mark.parametrize("degree", [2, 3, 4, 5, 6])
def test_equioscillation(name, interval, degree):
    """Chebyshev alternation: p+2 points where the error alternates in sign with
    equal magnitude eps, and eps is the maximum over the whole interval."""
    a, b = interval
    f = AP.TARGETS[name]
    fit = AP.fit(name, degree, a, b)
    e = R.equioscillation(f, fit)
    assert len(e) == degree + 2
    assert np.all(np.sign(e[1:]) == -np.sign(e[:-1]))
    np.testing.assert_allclose(np.abs(e), fit.eps, rtol=1e-6)
    assert R.max_error(f, fit, a, b, 400001) <= fit.eps * (1 + 1e-6)


@pytest.mark.parametrize("degree", [3, 5])
def test_equioscillation_oscillatory_target(degree):
    """cos(12 z) on [0, 1], a target with nearly two periods on the
    interval: the fit alternates p + 2 times at the level, and the level is
    the maximum error over the interval."""
    f = lambda z: np.cos(12.0 * np.asarray(z, dtype=np.float64))  # noqa: E731
    fit = R.remez(f, 0.0, 1.0, degree)
    e = R.equioscillation(f, fit)
    assert len(e) == degree + 2
    assert np.all(np.sign(e[1:]) == -np.sign(e[:-1]))
    np.testing.assert_allclose(np.abs(e), fit.eps, rtol=1e-6)
    assert R.max_error(f, fit, 0.0, 1.0, 400001) <= fit.eps * (1 + 1e-6)


@pytest.mark.parametrize("freq,degree", [(30.0, 3), (25.0, 4)])
def test_zero_polynomial_when_the_target_alternates(freq, degree):
    """cos(f z) on [0, 1] reaches +1 and -1 alternately at z = k pi / f, more
    than p + 2 times for these f: by Chebyshev's alternation theorem the
    zero polynomial is the best approximation and the level is exactly 1.
    The exchange meets more than p + 2 extrema on the way and must keep the
    p + 2 that contain the global maximum."""
    f = lambda z: np.cos(freq * np.asarray(z, dtype=np.float64))  # noqa: E731
    fit = R.remez(f, 0.0, 1.0, degree)
    assert fit.eps == pytest.approx(1.0, rel=1e-6)
    z = np.linspace(0.0, 1.0, 20001)
    assert np.max(np.abs(fit(z))) < 1e-6  # the zero polynomial, up to the exchange's tolerance


def test_degree_monotone():
    """More degrees of freedom never increase the minimax error."""
    for name, (a, b) in [("acos_lo", AP.ACOS_LO_INTERVAL), ("exp", (0.0, 10.0))]:
        eps = [AP.fit(name, d, a, b).eps for d in range(2, 7)]
        assert all(e2 < e1 for e1, e2 in zip(eps, eps[1:]))


@pytest.mark.parametrize("key,f", [("exp_rational", AP.f_expneg), ("ent_rational", AP.f_ent)])
def test_paper_rationals(golden, key, f):
    """The printed rationals, rounded to 7 digits, stay within 1.2x of the
    stated eps over their interval, and the oracle carries the same values."""
    g = golden[key]
    a, b = g["interval"]
    err = R.max_error(f, _rat(g["num"], g["den"]), a, b)
    assert g["eps"] * 0.9 <= err <= 1.2 * g["eps"]
    src = PT.EXP_RATIONAL_NUM if key == "exp_rational" else PT.ENT_RATIONAL_NUM
    assert src == g["num"]


def test_oracle_tables_match_golden(golden):
    assert PT.TABLE1_ARCSIN == golden["table1_arcsin"]["coef"]
    assert PT.TABLE1_ARCCOS == golden["table1_arccos"]["coef"]
    for d, row in golden["table2_exp"]["rows"].items():
        assert PT.TABLE2_EXP[int(d)][1] == row["coef"]
    assert PT.ENT_RATIONAL_DEN == golden["ent_rational"]["den"]
    assert PT.EXP_RATIONAL_DEN == golden["exp_rational"]["den"]


def test_exp_cutoff_value(golden):
    g = golden["exp_cutoff"]
    assert AP.f_expneg(g["T"]) == pytest.approx(g["exp_minus_T"], rel=2e-7)


def test_acos_identity():
    """Sec. 3.1: arccos z = 2 arcsin(sqrt(0.5 (1 - z))) = g(sqrt(1 - z))."""
    z = np.linspace(0.5, 1.0, 1001)
    np.testing.assert_allclose(AP.f_acos_hi(np.sqrt(1 - z)), np.arccos(z), atol=1e-14)


def test_piecewise_join():
    """The two Table 1 pieces meet at z = 0.5 within the sum of their errors."""
    lo, hi = AP.acos_pieces(4, "paper")
    jump = abs(lo(0.5) - hi(math.sqrt(0.5)))
    assert jump <= PT.TABLE1_ARCCOS_EPS + PT.TABLE1_ARCSIN_EPS + 1e-6


# ---------------------------------------------------------------- rational Remez

RATIONAL_CASES = [("exp_rational", "exp"), ("ent_rational", "ent")]


@pytest.mark.parametrize("key,fn", RATIONAL_CASES)
def test_rational_remez_reproduces_paper(golden, key, fn):
    """The oracle's own (4,4) rational Remez lands on the paper's minimax
    rationals (Sec. 3.2 tab_exp_rat, Sec. 3.3 tab_ent_rat): the stated eps to
    0.25 % (ours is 0.18 % lower for both functions), the printed
    coefficients (normalised to den[0] = 1) to 5e-4, and below the error of
    the printed, 7-digit coefficients themselves."""
    g = golden[key]
    a, b = g["interval"]
    r = R.rational_remez(AP.TARGETS[fn], a, b, 4, 4)
    assert r.eps == pytest.approx(g["eps"], rel=2.5e-3)
    printed = AP.Approximant(g["num"], g["den"])
    assert r.eps < R.max_error(AP.TARGETS[fn], printed, a, b)
    np.testing.assert_allclose(r.num, np.array(g["num"]) / g["den"][0], rtol=5e-4)
    np.testing.assert_allclose(r.den, np.array(g["den"]) / g["den"][0], rtol=5e-4)


@pytest.mark.parametrize("fn,interval", [("exp", (0.0, 10.0)), ("ent", (0.05, 1.0)),
                                         ("ent", (0.018, 1.0))])
@pytest.mark.parametrize("d", [2, 3, 4])
def test_rational_equioscillation(fn, interval, d):
    """Checked on a dense grid, independently of the exchange: the error of
    the best (d,d) rational alternates in sign on at least 2d + 2 extrema of
    magnitude eps (the characterisation of a non-degenerate best
    approximation), and the denominator has no zero on the interval."""
    a, b = interval
    r = R.rational_remez(AP.TARGETS[fn], a, b, d, d)
    z = np.linspace(a, b, 400001)
    q = np.polynomial.polynomial.polyval(z, r.den)
    assert np.all(q > 0.0)
    e = AP.TARGETS[fn](z) - r(z)
    assert np.max(np.abs(e)) == pytest.approx(r.eps, rel=1e-6)
    # extrema of runs of one sign reaching the level
    runs, cur = [], None
    for v in e[np.abs(e) > 0.999 * r.eps]:
        s = v > 0
        if cur is None or s != cur:
            runs.append(s)
            cur = s
    assert len(runs) >= 2 * d + 2


def test_rational_beats_polynomial_with_as_many_coefficients():
    """Sec. 3.2: the rational is the better form for EXP on [0, 10]: the
    (2,2) rational (5 coefficients) beats the degree-4 polynomial, the (4,4)
    one (9 coefficients) beats degree 8 by orders of magnitude."""
    f = AP.TARGETS["exp"]
    for d, pd in [(2, 4), (4, 8)]:
        assert R.rational_remez(f, 0.0, 10.0, d, d).eps < R.remez(f, 0.0, 10.0, pd).eps
    assert (R.rational_remez(f, 0.0, 10.0, 2, 2).eps > R.rational_remez(f, 0.0, 10.0, 3, 3).eps
            > R.rational_remez(f, 0.0, 10.0, 4, 4).eps)


def test_rational_remez_reduces_to_polynomial():
    """A (m, 0)-like case: the best rational of a polynomial of degree m is
    that polynomial (error at rounding level)."""
    def f(z):
        return 1.0 - 2.0 * np.asarray(z) + 0.5 * np.asarray(z) ** 2
    r = R.rational_remez(f, -1.0, 2.0, 2, 1)
    assert r.eps < 1e-12
