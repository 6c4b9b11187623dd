"""Filtering-quality criteria of Sec. 4, in FP64.

TEST INFRASTRUCTURE ONLY (oracle side).

  MAE(X, Y) = 1/(3MN) sum ||x - y||_1                     (Sec. 4, item 1)
  MSE(X, Y) = 1/(3MN) sum ||x - y||_2^2                   (Sec. 4, item 2)
  NCD(X, Y) = sum ||x^Lab - y^Lab||_2 / sum ||x^Lab||_2   (Sec. 4, item 3)
  PSNR      = 10 log10(255^2 / MSE)   (not in the paper; the dB figure used to
                                       judge an approximation's quality drop)

The paper names CIE L*a*b* without a conversion; the reading here is sRGB
(IEC 61966-2-1) linearisation, the sRGB primaries' D65 matrix, the D65 white
point of that matrix, and the CIE 1976 L*a*b* formulas.
"""
from __future__ import annotations

import numpy as np

_M = np.array([[0.4124, 0.3576, 0.1805],
               [0.2126, 0.7152, 0.0722],
               [0.0193, 0.1192, 0.9505]])
_WHITE = _M.sum(axis=1)  # XYZ of sRGB (1, 1, 1): the D65 white of the matrix


def _rgb(a):
    a = np.asarray(a)
    return a[..., :3].astype(np.float64)


def mae(x, y) -> float:
    return float(np.abs(_rgb(x) - _rgb(y)).sum(axis=-1).mean() / 3.0)


def mse(x, y) -> float:
    return float(((_rgb(x) - _rgb(y)) ** 2).sum(axis=-1).mean() / 3.0)


def psnr(x, y) -> float:
    m = mse(x, y)
    return float("inf") if m == 0.0 else float(10.0 * np.log10(255.0 ** 2 / m))


def srgb_to_lab(img) -> np.ndarray:
    c = _rgb(img) / 255.0
    lin = np.where(c <= 0.04045, c / 12.92, ((c + 0.055) / 1.055) ** 2.4)
    xyz = lin @ _M.T / _WHITE
    d = 6.0 / 29.0
    f = np.where(xyz > d ** 3, np.cbrt(xyz), xyz / (3.0 * d * d) + 4.0 / 29.0)
    L = 116.0 * f[..., 1] - 16.0
    a = 500.0 * (f[..., 0] - f[..., 1])
    b = 200.0 * (f[..., 1] - f[..., 2])
    return np.stack([L, a, b], axis=-1)


def ncd(x, y) -> float:
    lx, ly = srgb_to_lab(x), srgb_to_lab(y)
    num = np.sqrt(((lx - ly) ** 2).sum(axis=-1)).sum()
    den = np.sqrt((lx ** 2).sum(axis=-1)).sum()
    return float(num / den)


def changed_fraction(a, b) -> float:
    """Fraction of pixels whose RGB output differs."""
    return float(np.any(_rgb(a) != _rgb(b), axis=-1).mean())
