"""ctypes front end of the FP64 C oracle (oracle/vfo.c).

TEST INFRASTRUCTURE ONLY.  Builds oracle/vfo.c with gcc on first use (or from
the package's build step) and runs the whole-image filters of Sec. 3 with the
approximants of oracle.approximants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import approximants as AP
from . import paper_tables as T

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vfo.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libvfo.so")
_lock = threading.Lock()
_lib = None

CRITERIA = {"vmf": 0, "bvdf": 1, "amnfe": 2, "amnfg": 3, "evmf": 4, "evbdf": 5}
APPROX = {"exact": 0, "poly": 1, "rational": 2, "rational_fit": 2}  # C side: any rational
MAXC = 16


class _Approximant(ctypes.Structure):
    _fields_ = [("num_len", ctypes.c_int), ("den_len", ctypes.c_int),
                ("num", ctypes.c_double * MAXC), ("den", ctypes.c_double * MAXC)]


class _Params(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int), ("criterion", ctypes.c_int),
                ("approx", ctypes.c_int), ("kappa", ctypes.c_double),
                ("exp_cutoff", ctypes.c_double), ("ent_cutoff", ctypes.c_double),
                ("acos_lo", _Approximant), ("acos_hi", _Approximant),
                ("expo", _Approximant), ("ent", _Approximant)]


class _Diag(ctypes.Structure):
    _fields_ = [("sel", ctypes.c_void_p), ("gap", ctypes.c_void_p),
                ("sw", ctypes.c_void_p), ("yreal", ctypes.c_void_p)]


def build(force: bool = False) -> str:
    """Compile vfo.c into oracle/_build/libvfo.so (plain IEEE FP64: no fast
    math, no FMA contraction, so x86 and Arm hosts agree)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            _lib.vfo_filter.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P,
                                        ctypes.c_int]
            _lib.vfo_filter_rows.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                             P, P, ctypes.c_int, ctypes.c_int]
            _lib.vfo_window_aggregates.argtypes = [P, ctypes.c_int, P, P]
            _lib.vfo_window_evmf_switch.argtypes = [P, ctypes.c_int, P, P]
            _lib.vfo_window_amnf.argtypes = [P, ctypes.c_int, P, P]
            for name in ("vfo_angle_exact", "vfo_angle_acos"):
                getattr(_lib, name).argtypes = [P, P]
                getattr(_lib, name).restype = ctypes.c_double
            _lib.vfo_angle_approx.argtypes = [P, P, P]
            _lib.vfo_angle_approx.restype = ctypes.c_double
            _lib.vfo_expneg.argtypes = [P, ctypes.c_double]
            _lib.vfo_expneg.restype = ctypes.c_double
            _lib.vfo_ent.argtypes = [P, ctypes.c_double]
            _lib.vfo_ent.restype = ctypes.c_double
        return _lib


def _fill(dst: _Approximant, a: AP.Approximant):
    dst.num_len = len(a.num)
    dst.den_len = len(a.den)
    for k, v in enumerate(a.num):
        dst.num[k] = v
    for k, v in enumerate(a.den):
        dst.den[k] = v


class Config:
    """One filter configuration: criterion, window, approximation, degree and
    the paper's constants (kappa, EXP and ENT cut-offs)."""

    def __init__(self, criterion: str, window: int = 3, approx: str = "exact",
                 degree: int = 4, kappa: float = T.KAPPA, exp_cutoff: float = T.EXP_CUTOFF,
                 ent_cutoff: float | None = None, coeffs: str = "fit"):
        if criterion not in CRITERIA:
            raise ValueError(criterion)
        if approx not in APPROX:
            raise ValueError(approx)
        n = window * window
        self.criterion, self.window, self.approx, self.degree = criterion, window, approx, degree
        self.kappa, self.exp_cutoff = float(kappa), float(exp_cutoff)
        self.ent_cutoff = float(AP.default_ent_cutoff(n) if ent_cutoff is None else ent_cutoff)
        self.coeffs = coeffs
        p = _Params()
        p.window, p.criterion, p.approx = window, CRITERIA[criterion], APPROX[approx]
        p.kappa, p.exp_cutoff, p.ent_cutoff = self.kappa, self.exp_cutoff, self.ent_cutoff
        if approx != "exact":
            if criterion in ("bvdf", "evbdf"):
                if approx != "poly":
                    raise ValueError("the paper gives no rational for arccos")
                lo, hi = AP.acos_pieces(degree, coeffs)
                _fill(p.acos_lo, lo)
                _fill(p.acos_hi, hi)
                if criterion == "evbdf":  # the switch's ENT polynomial, same degree
                    _fill(p.ent, AP.ent_approximant(approx, degree, self.ent_cutoff))
            elif criterion in ("amnfe", "amnfg"):
                _fill(p.expo, AP.exp_approximant(approx, degree, self.exp_cutoff, coeffs))
            elif criterion == "evmf":
                _fill(p.ent, AP.ent_approximant(approx, degree, self.ent_cutoff))
            # VMF has no elementary function to approximate (Sec. 3.3 keeps the
            # Euclidean median exact): the approximation flag is ignored.
        self.params = p

    def ptr(self):
        return ctypes.byref(self.params)


def filter_image(img: np.ndarray, cfg: Config, threads: int = 1, rows=None):
    """Filter an H x W x C uint8 image (C = 3 or 4).  Returns (out, diag) where
    diag holds per-pixel 'sel', 'gap', 'sw' and (AMNF) 'yreal'.  With rows=(r0, r1)
    only those output rows are computed (the others stay zero)."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    if img.ndim != 3 or img.shape[2] not in (3, 4):
        raise ValueError("expected H x W x 3 or H x W x 4 uint8")
    H, W, C = img.shape
    out = np.zeros_like(img)
    sel = np.full((H, W), -1, dtype=np.int32)
    gap = np.full((H, W), np.inf, dtype=np.float64)
    sw = np.zeros((H, W), dtype=np.uint8)
    yreal = np.zeros((H, W, 3), dtype=np.float64)
    d = _Diag(sel.ctypes.data, gap.ctypes.data, sw.ctypes.data, yreal.ctypes.data)
    L = lib()
    if rows is None:
        rc = L.vfo_filter(img.ctypes.data, H, W, C, ctypes.addressof(cfg.params), out.ctypes.data,
                          ctypes.addressof(d), int(threads))
    else:
        rc = L.vfo_filter_rows(img.ctypes.data, H, W, C, ctypes.addressof(cfg.params),
                               out.ctypes.data, ctypes.addressof(d), int(rows[0]), int(rows[1]))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return out, {"sel": sel, "gap": gap, "sw": sw, "yreal": yreal}


def window_aggregates(cfg: Config, xs: np.ndarray) -> np.ndarray:
    xs = np.ascontiguousarray(xs, dtype=np.float64).reshape(-1, 3)
    agg = np.zeros(len(xs))
    lib().vfo_window_aggregates(ctypes.addressof(cfg.params), len(xs), xs.ctypes.data,
                                agg.ctypes.data)
    return agg


def window_evmf_switch(cfg: Config, xs: np.ndarray):
    xs = np.ascontiguousarray(xs, dtype=np.float64).reshape(-1, 3)
    gap = ctypes.c_double(0.0)
    s = lib().vfo_window_evmf_switch(ctypes.addressof(cfg.params), len(xs), xs.ctypes.data,
                                     ctypes.addressof(gap))
    return bool(s), gap.value


def window_amnf(cfg: Config, xs: np.ndarray) -> np.ndarray:
    xs = np.ascontiguousarray(xs, dtype=np.float64).reshape(-1, 3)
    y = np.zeros(3)
    lib().vfo_window_amnf(ctypes.addressof(cfg.params), len(xs), xs.ctypes.data, y.ctypes.data)
    return y


def angle(a, b, form: str = "exact", cfg: Config | None = None) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    L = lib()
    if form == "exact":
        return L.vfo_angle_exact(a.ctypes.data, b.ctypes.data)
    if form == "acos":
        return L.vfo_angle_acos(a.ctypes.data, b.ctypes.data)
    return L.vfo_angle_approx(ctypes.addressof(cfg.params), a.ctypes.data, b.ctypes.data)


def expneg(cfg: Config, z: float) -> float:
    return lib().vfo_expneg(ctypes.addressof(cfg.params), float(z))


def ent(cfg: Config, z: float) -> float:
    return lib().vfo_ent(ctypes.addressof(cfg.params), float(z))
