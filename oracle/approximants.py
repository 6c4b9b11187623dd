"""Target functions of Sec. 3 and the approximants the oracle substitutes.

TEST INFRASTRUCTURE ONLY (oracle side).

  acos_lo : arccos(z) on [0, 0.5]                       (Table 1, ARCCOS row)
  acos_hi : g(tau) = 2 arcsin(tau / sqrt 2) on [0, 1/sqrt 2]  (Table 1, ARCSIN)
  exp     : exp(-z) on [0, T], T = 10                   (Table 2, tab_exp_rat)
  ent     : z ln z on [T, 1], T = 0.05                  (tab_ent_rat)

Polynomials of degree 2..6 come from the oracle's own Remez fit (oracle.remez);
'rational' is the paper's printed (4,4) rational (oracle.paper_tables),
'rational_fit' the oracle's own best (d,d) rational (oracle.remez.rational_remez)
on the filter's interval.
"""
from __future__ import annotations

import functools
import math

import numpy as np

from . import paper_tables as T
from .remez import rational_remez, remez


def f_acos(z):
    return np.arccos(z)


def f_acos_hi(tau):
    """Sec. 3.1: arccos(z) = 2 arcsin(tau / sqrt 2) with tau = sqrt(1 - z)."""
    return 2.0 * np.arcsin(np.asarray(tau) / math.sqrt(2.0))


def f_expneg(z):
    return np.exp(-np.asarray(z, dtype=np.float64))


def f_ent(z):
    """Sec. 3.3: ENT(z) = z log z, natural log (0 log 0 = 0)."""
    z = np.asarray(z, dtype=np.float64)
    return np.where(z > 0.0, z * np.log(np.where(z > 0.0, z, 1.0)), 0.0)


ACOS_LO_INTERVAL = (0.0, 0.5)
ACOS_HI_INTERVAL = (0.0, 1.0 / math.sqrt(2.0))

TARGETS = {
    "acos_lo": f_acos,
    "acos_hi": f_acos_hi,
    "exp": f_expneg,
    "ent": f_ent,
}


@functools.lru_cache(maxsize=None)
def fit(name: str, degree: int, lo: float, hi: float):
    """Degree-`degree` minimax polynomial of TARGETS[name] on [lo, hi]."""
    return remez(TARGETS[name], lo, hi, degree)


@functools.lru_cache(maxsize=None)
def rational_fit(name: str, degree: int, lo: float, hi: float):
    """Best (degree, degree) rational of TARGETS[name] on [lo, hi]."""
    return rational_remez(TARGETS[name], lo, hi, degree, degree)


def default_ent_cutoff(n: int) -> float:
    """ENT cut-off.  Sec. 3.3 fixes T = 0.05 for the paper's windows (n = 9,
    where the mean P_i is 1/9).  For larger windows the mean P_i = 1/n falls
    below 0.05 and most terms would be cut; the cut-off is scaled with the
    mean, T_n = 0.05 * 9 / n (a reading: the paper only studies n = 9)."""
    return T.ENT_CUTOFF if n <= 9 else T.ENT_CUTOFF * 9.0 / n


class Approximant:
    """p(z) or p(z)/q(z), coefficients in increasing powers."""

    def __init__(self, num, den=None):
        self.num = [float(v) for v in num]
        self.den = [float(v) for v in den] if den is not None else []

    def __call__(self, z):
        z = np.asarray(z, dtype=np.float64)
        p = np.polynomial.polynomial.polyval(z, self.num)
        if not self.den:
            return p
        return p / np.polynomial.polynomial.polyval(z, self.den)


def acos_pieces(degree: int, source: str = "fit"):
    """The two BVDF pieces (Sec. 3.1).  source='paper' takes the printed
    Table 1 values (degree 4 only)."""
    if source == "paper":
        if degree != 4:
            raise ValueError("Table 1 prints degree 4 only")
        return Approximant(T.TABLE1_ARCCOS), Approximant(T.TABLE1_ARCSIN)
    lo = fit("acos_lo", degree, *ACOS_LO_INTERVAL)
    hi = fit("acos_hi", degree, *ACOS_HI_INTERVAL)
    return Approximant(lo.coef), Approximant(hi.coef)


def exp_approximant(kind: str, degree: int, cutoff: float = T.EXP_CUTOFF,
                    source: str = "fit"):
    """EXP approximant on [0, cutoff] (Sec. 3.2)."""
    if kind == "rational_fit":
        r = rational_fit("exp", degree, 0.0, float(cutoff))
        return Approximant(r.num, r.den)
    if kind == "rational":
        if cutoff != T.EXP_CUTOFF:
            raise ValueError("the paper's EXP rational is fitted on [0, 10]")
        return Approximant(T.EXP_RATIONAL_NUM, T.EXP_RATIONAL_DEN)
    if source == "paper":
        return Approximant(T.TABLE2_EXP[degree][1])
    return Approximant(fit("exp", degree, 0.0, float(cutoff)).coef)


def ent_approximant(kind: str, degree: int, cutoff: float = T.ENT_CUTOFF):
    """ENT approximant on [cutoff, 1] (Sec. 3.3).  The rational is the paper's,
    fitted on [0.05, 1]; below 0.05 (larger windows) it is used as printed.
    The own rational fit is made on [cutoff, 1]."""
    if kind == "rational_fit":
        r = rational_fit("ent", degree, float(cutoff), 1.0)
        return Approximant(r.num, r.den)
    if kind == "rational":
        return Approximant(T.ENT_RATIONAL_NUM, T.ENT_RATIONAL_DEN)
    return Approximant(fit("ent", degree, float(cutoff), 1.0).coef)
