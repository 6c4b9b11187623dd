"""Pins of the oracle's approximant evaluation: the EXP and ENT functions of
the C oracle (oracle/vfo.c, `vfo_expneg`, `vfo_ent`, `vfo_eval_approximant`)
evaluated through `oracle.filters`, against exp(-z) and z ln z themselves and
against the error levels the paper prints (Sec. 3.2 Table 2 and tab_exp_rat,
Sec. 3.3 tab_ent_rat).  CPU only.

What each test catches: a rational evaluated as anything but p(z)/q(z), an
argument scaled or shifted before the approximant, an approximant scaled
after it, a cut-off applied on the wrong side, a polynomial of the wrong
degree or interval.  The minimax level of each approximant is attained, so
every check bounds the maximum error from both sides.
"""
import math

import numpy as np
import pytest

from oracle import approximants as AP
from oracle import filters as F
from oracle import paper_tables as PT

# Degree 5 and 6 levels of exp(-z) on [0, 10] and degree 2..6 levels of
# z ln z on [0.05, 1], computed once with an independent FP64 Remez script
# (not the oracle's); Table 2 prints degrees 2..4 of exp(-z).
EXP_LEVEL_EXTRA = {5: 1.188e-2, 6: 3.763e-3}
ENT_LEVEL = {2: 2.82e-2, 3: 8.96e-3, 4: 3.43e-3, 5: 1.46e-3, 6: 6.66e-4}


def _max_err_exp(cfg, lo, hi, n=40001):
    z = np.linspace(lo, hi, n)
    got = np.array([F.expneg(cfg, v) for v in z])
    return float(np.max(np.abs(got - np.exp(-z))))


def _max_err_ent(cfg, lo, hi, n=40001):
    z = np.linspace(lo, hi, n)
    got = np.array([F.ent(cfg, v) for v in z])
    return float(np.max(np.abs(got - z * np.log(z))))


# ---------------------------------------------------------------- EXP (Sec. 3.2)


@pytest.mark.parametrize("degree", [2, 3, 4])
@pytest.mark.parametrize("coeffs", ["fit", "paper"])
def test_exp_poly_level_table2(golden, degree, coeffs):
    """The degree-2..4 EXP polynomials (the oracle's own fit and the printed
    Table 2 rows) are within the printed eps of exp(-z) on [0, 10], and reach
    it (a minimax error is attained)."""
    eps = golden["table2_exp"]["rows"][str(degree)]["eps"]
    cfg = F.Config("amnfe", 3, "poly", degree, coeffs=coeffs)
    err = _max_err_exp(cfg, 0.0, PT.EXP_CUTOFF)
    assert eps * (1 - 2e-3) <= err <= eps * (1 + 2e-3)


@pytest.mark.parametrize("degree", [5, 6])
def test_exp_poly_level_high_degrees(degree):
    eps = EXP_LEVEL_EXTRA[degree]
    err = _max_err_exp(F.Config("amnfe", 3, "poly", degree), 0.0, PT.EXP_CUTOFF)
    assert eps * (1 - 2e-3) <= err <= eps * (1 + 2e-3)


def test_exp_paper_rational_level(golden):
    """tab_exp_rat: the printed (4,4) rational through the C evaluation, within
    1.2 x the printed eps of exp(-z) on [0, 10] and not far below it."""
    eps = golden["exp_rational"]["eps"]
    err = _max_err_exp(F.Config("amnfe", 3, "rational"), 0.0, PT.EXP_CUTOFF)
    assert 0.9 * eps <= err <= 1.2 * eps


@pytest.mark.parametrize("key,kind,f,lo,hi", [
    ("exp_rational", "exp", lambda z: np.exp(-z), 0.0, 10.0),
    ("ent_rational", "ent", lambda z: z * np.log(z), 0.05, 1.0)])
def test_paper_rationals_through_python_approximant(golden, key, kind, f, lo, hi):
    """The printed (4,4) rationals (tab_exp_rat, tab_ent_rat) evaluated by the
    oracle's Python `Approximant` (the coefficients the C oracle and the GPU
    tests receive): within [0.9, 1.2] x the printed eps of the target."""
    ap = AP.exp_approximant("rational", 4) if kind == "exp" else AP.ent_approximant("rational", 4)
    z = np.linspace(lo, hi, 40001)
    err = float(np.max(np.abs(ap(z) - f(z))))
    eps = golden[key]["eps"]
    assert 0.9 * eps <= err <= 1.2 * eps


def test_acos_pieces_are_table1(golden):
    """The BVDF pieces the filters receive (`acos_pieces`, degree 4, the
    oracle's own fit) are Table 1's rows: the same intervals, coefficients to
    the printed digits, and the pieces within their printed eps of arccos on
    each side of z = 0.5 (Sec. 3.1)."""
    assert AP.ACOS_LO_INTERVAL == pytest.approx(tuple(golden["table1_arccos"]["interval"]))
    assert AP.ACOS_HI_INTERVAL == pytest.approx(tuple(golden["table1_arcsin"]["interval"]))
    lo, hi = AP.acos_pieces(4)
    np.testing.assert_allclose(lo.num, golden["table1_arccos"]["coef"], rtol=2e-5, atol=2e-10)
    np.testing.assert_allclose(hi.num, golden["table1_arcsin"]["coef"], rtol=2e-5, atol=2e-10)
    z = np.linspace(0.0, 0.5, 20001)
    assert np.max(np.abs(lo(z) - np.arccos(z))) <= golden["table1_arccos"]["eps"] * 1.001
    z = np.linspace(0.5, 1.0, 20001)
    assert np.max(np.abs(hi(np.sqrt(1.0 - z)) - np.arccos(z))) <= (
        golden["table1_arcsin"]["eps"] * 1.001)


@pytest.mark.parametrize("degree", [2, 3, 4])
def test_exp_own_rational_level(degree):
    """The oracle's own (d,d) rational: its levelled error is attained by the C
    evaluation; the (4,4) one is no worse than the printed eps."""
    r = AP.rational_fit("exp", degree, 0.0, PT.EXP_CUTOFF)
    err = _max_err_exp(F.Config("amnfe", 3, "rational_fit", degree), 0.0, PT.EXP_CUTOFF)
    assert r.eps * (1 - 1e-3) <= err <= r.eps * (1 + 1e-3)
    if degree == 4:
        assert err <= PT.EXP_RATIONAL_EPS


@pytest.mark.parametrize("approx,degree", [("exact", 0), ("poly", 4), ("rational", 4),
                                           ("rational_fit", 3)])
def test_exp_zero_outside_cutoff(approx, degree):
    """E = 0 for arguments outside [0, T] (Sec. 3.2), for every variant; at
    z = T itself the function is still evaluated (e^-10 = 4.539993e-05)."""
    cfg = F.Config("amnfe", 3, approx, max(degree, 2))
    for z in (-1e-9, -1.0, PT.EXP_CUTOFF * (1 + 1e-12), 10.5, 1e3):
        assert F.expneg(cfg, z) == 0.0
    v = F.expneg(cfg, PT.EXP_CUTOFF)
    tol = {"exact": 1e-12, "poly": 3.4e-2, "rational": 2.7e-6, "rational_fit": 1e-3}[approx]
    assert abs(v - PT.EXP_AT_CUTOFF) <= tol
    if approx == "exact":
        assert v == pytest.approx(PT.EXP_AT_CUTOFF, rel=1e-6)


def test_exp_cutoff_moves_interval():
    """A non-default cut-off refits the polynomial on [0, T'] and zeroes E
    above T': the error level of the fit on the shorter interval is attained
    there (degree 4 on [0, n^(kappa/3)], the argument bound of a 5 x 5
    window)."""
    T = 25 ** (0.33 / 3)
    cfg = F.Config("amnfe", 5, "poly", 4, exp_cutoff=T)
    eps = AP.fit("exp", 4, 0.0, T).eps
    assert eps < 1e-4
    err = _max_err_exp(cfg, 0.0, T)
    assert eps * (1 - 1e-3) <= err <= eps * (1 + 1e-3)
    assert F.expneg(cfg, T * 1.001) == 0.0


# ---------------------------------------------------------------- ENT (Sec. 3.3)


@pytest.mark.parametrize("degree", [2, 3, 4, 5, 6])
def test_ent_poly_level(degree):
    """The ENT polynomials on [0.05, 1] reach their minimax level of z ln z."""
    eps = ENT_LEVEL[degree]
    err = _max_err_ent(F.Config("evmf", 3, "poly", degree), PT.ENT_CUTOFF, 1.0)
    assert eps * (1 - 1e-2) <= err <= eps * (1 + 1e-2)


@pytest.mark.parametrize("w", [5, 7])
def test_ent_poly_level_scaled_cutoff(w):
    """For n > 9 the ENT polynomial is refitted on [T_n, 1], T_n = 0.05 * 9 / n;
    the C evaluation attains that fit's level there and is 0 below T_n."""
    T = AP.default_ent_cutoff(w * w)
    assert T == pytest.approx(0.45 / (w * w))
    cfg = F.Config("evmf", w, "poly", 4)
    eps = AP.fit("ent", 4, T, 1.0).eps
    err = _max_err_ent(cfg, T, 1.0)
    assert eps * (1 - 1e-3) <= err <= eps * (1 + 1e-3)
    assert F.ent(cfg, T * (1 - 1e-9)) == 0.0


def test_ent_paper_rational_level(golden):
    """tab_ent_rat: the printed (4,4) rational within 1.2 x the printed eps of
    z ln z on [0.05, 1], and not far below it."""
    eps = golden["ent_rational"]["eps"]
    err = _max_err_ent(F.Config("evmf", 3, "rational"), PT.ENT_CUTOFF, 1.0)
    assert 0.9 * eps <= err <= 1.2 * eps


def test_ent_paper_rational_below_interval():
    """Below 0.05 (the 5 x 5 and 7 x 7 cut-offs) the printed rational is used
    as printed: its error there stays below 1.7e-3."""
    T = AP.default_ent_cutoff(49)
    err = _max_err_ent(F.Config("evmf", 7, "rational"), T, PT.ENT_CUTOFF)
    assert err <= 1.7e-3


@pytest.mark.parametrize("degree", [2, 3, 4])
def test_ent_own_rational_level(degree):
    r = AP.rational_fit("ent", degree, PT.ENT_CUTOFF, 1.0)
    err = _max_err_ent(F.Config("evmf", 3, "rational_fit", degree), PT.ENT_CUTOFF, 1.0)
    assert r.eps * (1 - 1e-3) <= err <= r.eps * (1 + 1e-3)
    if degree == 4:
        assert err <= PT.ENT_RATIONAL_EPS


@pytest.mark.parametrize("approx", ["exact", "poly", "rational", "rational_fit"])
def test_ent_zero_below_cutoff(approx):
    cfg = F.Config("evmf", 3, approx, 4)
    for z in (0.0, 1e-6, 0.01, PT.ENT_CUTOFF * (1 - 1e-12)):
        assert F.ent(cfg, z) == 0.0
    assert F.ent(cfg, 1.0) == pytest.approx(0.0, abs=4e-3)
    assert F.ent(cfg, 0.5) == pytest.approx(0.5 * math.log(0.5), abs=4e-3)


# ---------------------------------------------------------------- the filters


def _amnf_two_value(crit, k, E):
    """AMNF on a window of n - k samples a (incl. the centre) and k samples b
    (Sec. 3.2, Eq. equ_amnf): h_a = n^(-kappa/3) k d1, h_b = n^(-kappa/3)
    (n - k) d1; a-weights h_a^-3 E(0), b-weights h_b^-3 E(z_b); a two-point
    weighted mean."""
    n, kappa = 9, PT.KAPPA
    a = np.array([100.0, 120.0, 90.0])
    b = np.array([160.0, 30.0, 200.0])
    xs = np.tile(a, (n, 1))
    xs[[0, 2, 8][:k]] = b
    d1, d2 = np.abs(a - b).sum(), np.sqrt(((a - b) ** 2).sum())
    s = n ** (-kappa / 3)
    ha, hb = s * k * d1, s * (n - k) * d1
    zb = d1 / hb if crit == "amnfe" else 0.5 * (d2 / hb) ** 2
    wa, wb = ha ** -3 * E(0.0), hb ** -3 * E(zb)
    return xs, ((n - k) * wa * a + k * wb * b) / ((n - k) * wa + k * wb)


@pytest.mark.parametrize("crit", ["amnfe", "amnfg"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_amnf_two_value_with_paper_rational(crit, k):
    """The two-point closed form with E = the printed tab_exp_rat rational
    (typed-in coefficients evaluated here by numpy) equals the oracle's
    weighted mean; E(0) of the rational is num[0] / den[0], not 1."""
    P = np.polynomial.polynomial

    def E(z):
        return P.polyval(z, PT.EXP_RATIONAL_NUM) / P.polyval(z, PT.EXP_RATIONAL_DEN)

    xs, y = _amnf_two_value(crit, k, E)
    got = F.window_amnf(F.Config(crit, 3, "rational"), xs)
    np.testing.assert_allclose(got, y, rtol=1e-13)
    # and it differs from the exact kernel's output by the rational's error only
    _, yx = _amnf_two_value(crit, k, lambda z: math.exp(-z))
    assert np.max(np.abs(got - yx)) < 1e-3


@pytest.mark.parametrize("crit", ["amnfe", "amnfg"])
@pytest.mark.parametrize("degree", [2, 3, 4])
def test_amnf_two_value_with_table2(crit, degree):
    """The same closed form with E = the printed Table 2 polynomial."""
    c = PT.TABLE2_EXP[degree][1]

    def E(z):
        return np.polynomial.polynomial.polyval(z, c)

    xs, y = _amnf_two_value(crit, 2, E)
    got = F.window_amnf(F.Config(crit, 3, "poly", degree, coeffs="paper"), xs)
    np.testing.assert_allclose(got, y, rtol=1e-12)


def _switch_closed_form(xs, ENT):
    """EVMF switch (Sec. 3.3, Eq. equ_evf): P_i = r_i / sum r, beta_C =
    ENT(P_C) / sum_j ENT(P_j); filter iff P_C > beta_C.  Returns (switch,
    relative margin)."""
    mean = xs.mean(0)
    r = np.sqrt(((xs - mean) ** 2).sum(1))
    P = r / r.sum()
    e = np.array([ENT(p) for p in P])
    if e.sum() == 0.0:
        return False, np.inf
    beta = e[len(xs) // 2] / e.sum()
    pc = P[len(xs) // 2]
    return pc > beta, abs(pc - beta) / max(abs(pc), abs(beta), 1e-300)


@pytest.mark.parametrize("approx", ["rational", "poly"])
def test_evmf_switch_with_approximant(approx):
    """The EVMF switch with ENT replaced by the approximant (the printed
    tab_ent_rat rational, or the degree-3 polynomial fit on [0.05, 1]),
    evaluated here by numpy from its coefficients, agrees with the oracle on
    random windows away from the decision boundary; with the degree-3
    polynomial the decisions differ from the exact ENT's on some windows, so
    the approximant is really the one evaluated."""
    T = PT.ENT_CUTOFF
    if approx == "rational":
        num, den = PT.ENT_RATIONAL_NUM, PT.ENT_RATIONAL_DEN
    else:
        num, den = list(AP.fit("ent", 3, T, 1.0).coef), None
    P = np.polynomial.polynomial

    def ENT(z):
        if z < T or z <= 0.0:
            return 0.0
        v = P.polyval(z, num)
        return v / P.polyval(z, den) if den else v

    def ENTx(z):
        return z * math.log(z) if z >= T and z > 0.0 else 0.0

    cfg = F.Config("evmf", 3, approx, 3)
    rng = np.random.default_rng(21)
    agree = differ = 0
    for _ in range(3000):
        xs = rng.integers(0, 256, size=(9, 3)).astype(np.float64)
        if rng.random() < 0.7:
            xs[:] = xs[0] + rng.integers(-12, 13, size=(9, 3))
            xs[rng.integers(9)] = rng.integers(0, 256, 3)
        xs = np.clip(xs, 0, 255)
        expect, margin = _switch_closed_form(xs, ENT)
        got, _ = F.window_evmf_switch(cfg, xs)
        if margin > 1e-9:
            assert got == expect
            agree += 1
        ex, mx = _switch_closed_form(xs, ENTx)
        if mx > 1e-9 and margin > 1e-9 and ex != expect:
            differ += 1
    assert agree > 2900
    if approx == "poly":
        assert differ > 0


def test_bvdf_paper_table1_angle():
    """BVDF with the printed Table 1 pair: the approximate angle through the C
    evaluation is within the printed eps of the pieces (max of the two rows,
    plus the join) of the exact angle, on both sides of z = 0.5, and it
    equals the numpy evaluation of the printed rows (the printed coefficients
    are rounded to 7 digits, which moves the level by up to 2 % of eps)."""
    cfg = F.Config("bvdf", 3, "poly", 4, coeffs="paper")
    P = np.polynomial.polynomial
    eps = max(PT.TABLE1_ARCCOS_EPS, PT.TABLE1_ARCSIN_EPS)
    rng = np.random.default_rng(4)
    lo = hi = 0
    for _ in range(2000):
        a, b = rng.integers(1, 256, 3), rng.integers(1, 256, 3)
        z = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        z = min(max(z, 0.0), 1.0)
        got = F.angle(a, b, "approx", cfg)
        if z < 0.5:
            lo += 1
            ref = P.polyval(z, PT.TABLE1_ARCCOS)
        else:
            hi += 1
            ref = P.polyval(math.sqrt(1.0 - z), PT.TABLE1_ARCSIN)
        assert got == pytest.approx(ref, abs=1e-12)
        assert abs(got - F.angle(a, b)) <= eps * 1.03
    assert lo > 10 and hi > 10
