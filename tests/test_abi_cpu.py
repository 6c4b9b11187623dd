"""The C-ABI library builds, loads and exports every entry point its header
declares; argument checks that need no GPU.  CPU only."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(vf_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def vf():
    from paper_1009_0959_gb300 import build
    build.build()
    from paper_1009_0959_gb300 import vfilt
    return vfilt


def test_exports_every_declared_symbol(vf):
    L = vf.lib()
    declared = _declared()
    assert len(declared) >= 7
    for name in declared:
        assert hasattr(L, name), name


def test_status_strings(vf):
    assert vf.status_string(0) == "ok"
    assert "overlap" in vf.status_string(2)


def test_argument_errors_without_gpu(vf):
    """Rejected before any CUDA call: null pointers, bad sizes and enums,
    overlapping ranges, unsupported windows."""
    buf = (ctypes.c_uint8 * 4096)()
    base = ctypes.addressof(buf)
    assert vf.filter_ptr(0, base, 4, 4, 4, 16, 16) == 1                  # null input
    assert vf.filter_ptr(base, base + 2048, 0, 4, 4, 16, 16) == 1        # height 0
    assert vf.filter_ptr(base, base + 2048, 4, 4, 5, 20, 20) == 1        # channels 5
    assert vf.filter_ptr(base, base + 2048, 4, 4, 4, 8, 16) == 1         # pitch too small
    assert vf.filter_ptr(base, base + 8, 4, 4, 4, 16, 16) == 2           # overlap
    assert vf.filter_ptr(base, base + 2048, 4, 4, 4, 16, 16, window=9) == 3
    assert vf.filter_ptr(base, base + 2048, 4, 4, 4, 16, 16, window=4) == 1
    assert vf.filter_ptr(base, base + 2048, 4, 4, 4, 16, 16, criterion=7) == 1
    assert vf.filter_ptr(base, base + 2048, 4, 4, 4, 16, 16, criterion="bvdf",
                         approx="rational") == 3
    assert vf.filter_ptr(base, base + 2048, 4, 4, 4, 16, 16, criterion="bvdf", approx="poly",
                         degree=9) == 1
    assert vf.filter_ptr(base, base + 2048, 4, 4, 4, 16, 16, criterion="amnfe",
                         approx="rational", exp_cutoff=2.0) == 3


def test_image_too_large_rejected_without_gpu(vf):
    """Images whose tile grid would pass 2^31 - 1 CTAs are refused on the host
    (VF_ERR_UNSUPPORTED) before any CUDA call: the per-window path (VMF,
    2^20 x 2^20) and the pair-reuse path (BVDF 5 x 5, 2^21 x 2^20).  The
    pointers are never dereferenced; they only have to be distinct ranges."""
    w = 1 << 20
    a, b = 1 << 40, 1 << 46
    assert vf.filter_ptr(a, b, 1 << 20, w, 4, 4 * w, 4 * w, criterion="vmf") == 3
    assert vf.filter_ptr(a, b, 1 << 21, w, 4, 4 * w, 4 * w, criterion="bvdf", window=5,
                         approx="poly", degree=4) == 3


def test_library_remez_matches_paper_table1(vf, golden):
    """The library's own fit (independent of the oracle's) reproduces the
    paper's Table 1 and Table 2 to the printed precision."""
    import numpy as np
    for key, fn in [("table1_arcsin", "acos_hi"), ("table1_arccos", "acos_lo")]:
        g = golden[key]
        num, den, eps = vf.get_approximant(fn, "poly", 4, *g["interval"])
        assert den == []
        assert eps == pytest.approx(g["eps"], rel=1e-4)
        np.testing.assert_allclose(num, g["coef"], rtol=2e-5, atol=2e-10)
    for d, row in golden["table2_exp"]["rows"].items():
        num, _, eps = vf.get_approximant("exp", "poly", int(d), 0.0, 10.0)
        assert eps == pytest.approx(row["eps"], rel=1e-4)
        np.testing.assert_allclose(num, row["coef"], rtol=1e-5)


def test_library_rationals_are_the_papers(vf, golden):
    for key, fn in [("exp_rational", "exp"), ("ent_rational", "ent")]:
        num, den, eps = vf.get_approximant(fn, "rational")
        assert num == golden[key]["num"] and den == golden[key]["den"]
        assert eps == golden[key]["eps"]


def test_options(vf):
    vf.set_option("pair_reuse", 0)
    vf.set_option("pair_reuse", 2)
    vf.set_option("pair_reuse", 1)
    with pytest.raises(vf.VFError):
        vf.set_option("pair_reuse", 3)
    vf.set_option("tile_rows", 8)
    vf.set_option("tile_rows", 4)
    with pytest.raises(vf.VFError):
        vf.set_option("tile_rows", 3)
    for engine in (0, 2, 1):
        vf.set_option("gate_tensor_cores", engine)
    with pytest.raises(vf.VFError):
        vf.set_option("gate_tensor_cores", 3)
    for permille in (1000, 150, 0):  # the gated filter's sparse-form limit
        vf.set_option("gated_sparse", permille)
    for bad in (-1, 1001):
        with pytest.raises(vf.VFError):
            vf.set_option("gated_sparse", bad)


@pytest.mark.parametrize("fn,interval", [("exp", (0.0, 10.0)), ("ent", (0.05, 1.0)),
                                         ("exp", (0.0, 1.534)), ("ent", (0.018, 1.0))])
def test_library_rational_remez_matches_oracle(vf, fn, interval):
    """The library's rational Remez (C++, fixed-point solve on the reference)
    and the oracle's (numpy, generalised eigenproblem) are written apart;
    they agree on eps and on the rational's values."""
    import numpy as np
    from oracle import approximants as AP
    from oracle import remez as R
    a, b = interval
    for d in (2, 3, 4):
        num, den, eps = vf.get_approximant(fn, "rational_fit", d, a, b)
        assert len(num) == d + 1 and len(den) == d + 1 and den[0] == 1.0
        r = R.rational_remez(AP.TARGETS[fn], a, b, d, d)
        if r.eps > 1e-10:
            assert eps == pytest.approx(r.eps, rel=1e-5)
        else:
            assert eps < 1e-10
        z = np.linspace(a, b, 10001)
        lib = np.polynomial.polynomial.polyval(z, num) / np.polynomial.polynomial.polyval(z, den)
        assert np.max(np.abs(lib - r(z))) <= 1e-3 * max(r.eps, 1e-9)


def test_library_rational_fit_errors(vf):
    with pytest.raises(vf.VFError):
        vf.get_approximant("exp", "rational_fit", 5, 0.0, 10.0)
    with pytest.raises(vf.VFError):
        vf.get_approximant("exp", "rational_fit", 3, 1.0, 1.0)


def test_evbdf_argument_checks(vf):
    """EVBDF: exact or polynomial, FP32, single-image calls only (checked on
    the host, before any launch; VF_ERR_UNSUPPORTED = 3)."""
    base = 1 << 20
    assert vf.filter_ptr(base, base + 4096, 8, 8, 4, 32, 32, criterion="evbdf",
                         approx="rational") == 3
    assert vf.filter_ptr(base, base + 4096, 8, 8, 4, 32, 32, criterion="evbdf", approx="poly",
                         precision="fp16x2") == 3


def test_set_coefficients_round_trip(vf, golden):
    """vf_set_coefficients: the printed Table 1 / Table 2 rows and tab_exp_rat
    (as a caller's rational) load into the context and come back from
    vf_get_approximant as given, with their maximum error on the interval
    measured by the library (the printed eps, to the printed precision); a
    cleared entry gives the library's own fit back."""
    import numpy as np
    try:
        for key, fn in [("table1_arcsin", "acos_hi"), ("table1_arccos", "acos_lo")]:
            g = golden[key]
            vf.set_coefficients(fn, "poly", 4, g["coef"], lo=g["interval"][0], hi=g["interval"][1])
            num, den, eps = vf.get_approximant(fn, "poly", 4, *g["interval"])
            assert num == g["coef"] and den == []
            assert eps == pytest.approx(g["eps"], rel=3e-2)
        for d, row in golden["table2_exp"]["rows"].items():
            vf.set_coefficients("exp", "poly", int(d), row["coef"], lo=0.0, hi=10.0)
            num, _, eps = vf.get_approximant("exp", "poly", int(d), 0.0, 10.0)
            assert num == row["coef"]
            assert eps == pytest.approx(row["eps"], rel=2e-3)
        r = golden["exp_rational"]
        vf.set_coefficients("exp", "rational_fit", 4, r["num"], r["den"], 0.0, 10.0)
        num, den, eps = vf.get_approximant("exp", "rational_fit", 4, 0.0, 10.0)
        assert num == r["num"] and den == r["den"]
        assert 0.9 * r["eps"] <= eps <= 1.2 * r["eps"]
    finally:
        for fn in ("acos_hi", "acos_lo"):
            vf.set_coefficients(fn, "poly", 4)
        for d in (2, 3, 4):
            vf.set_coefficients("exp", "poly", d)
        vf.set_coefficients("exp", "rational_fit", 4)
    num, _, _ = vf.get_approximant("acos_lo", "poly", 4, 0.0, 0.5)
    # the library's own fit again: a_2 = -1.42988e-2 (the printed -1.429899e-2
    # differs in the fifth digit)
    assert num[2] == pytest.approx(-1.4298809e-2, rel=2e-6)
    num, den, _ = vf.get_approximant("exp", "rational_fit", 4, 0.0, 10.0)
    assert den[0] == 1.0 and np.isfinite(num).all()


def test_set_coefficients_error_inside_the_interval(vf):
    """The maximum error the library reports for a caller's approximant is
    taken over the whole interval, not only near its ends: the zero
    polynomial of z ln z on [0.05, 1] errs most at z = 1/e, by exactly 1/e
    (a minimax fit errs most at the ends as well, so it cannot show this)."""
    import math
    try:
        vf.set_coefficients("ent", "poly", 2, [0.0, 0.0, 0.0], lo=0.05, hi=1.0)
        _, _, eps = vf.get_approximant("ent", "poly", 2, 0.05, 1.0)
        assert eps == pytest.approx(1.0 / math.e, rel=1e-7)
    finally:
        vf.set_coefficients("ent", "poly", 2)


def test_default_params_are_the_papers(vf):
    """kappa = 0.33 (Sec. 3.2, the recommended kernel-width factor), the EXP
    cut-off T = 10 (Sec. 3.2) and the ENT cut-off chosen per window (Sec. 3.3's
    T = 0.05 at n = 9: a negative value asks for it)."""
    import ctypes
    p = vf.Params()
    vf.lib().vf_default_params(ctypes.byref(p))  # the C defaults themselves
    assert p.kappa == pytest.approx(0.33)
    assert p.exp_cutoff == pytest.approx(10.0)
    assert p.ent_cutoff < 0.0


def test_set_coefficients_errors(vf):
    E = vf.VFError
    with pytest.raises(E) as e:
        vf.set_coefficients("exp", "poly", 4, [1.0, 2.0, 3.0], lo=0.0, hi=10.0)  # too few
    assert e.value.name == "VF_ERR_ARG"
    with pytest.raises(E) as e:
        vf.set_coefficients("exp", "poly", 7, [0.0] * 8, lo=0.0, hi=10.0)  # degree > 6
    assert e.value.name == "VF_ERR_ARG"
    with pytest.raises(E) as e:
        vf.set_coefficients("exp", "rational", 4, [1.0] * 5, [1.0] * 5, 0.0, 10.0)
    assert e.value.name == "VF_ERR_UNSUPPORTED"
    with pytest.raises(E) as e:  # denominator 1 - z/5 vanishes at z = 5
        vf.set_coefficients("exp", "rational_fit", 2, [1.0, 0.0, 0.0], [1.0, -0.2, 0.0], 0.0, 10.0)
    assert e.value.name == "VF_ERR_ARG"
    with pytest.raises(E) as e:  # a zero between sample points: the sign change tells
        vf.set_coefficients("exp", "rational_fit", 2, [1.0, 0.0, 0.0],
                            [1.0, -1.0 / 5.00003, 0.0], 0.0, 10.0)
    assert e.value.name == "VF_ERR_ARG"
    with pytest.raises(E) as e:
        vf.set_coefficients("ent", "poly", 2, [0.0, float("nan"), 0.0], lo=0.05, hi=1.0)
    assert e.value.name == "VF_ERR_ARG"
    with pytest.raises(E) as e:
        vf.set_coefficients("ent", "poly", 2, [0.0, 1.0, 0.0], lo=1.0, hi=0.05)
    assert e.value.name == "VF_ERR_ARG"
    # nothing was stored by the failed calls
    num, _, _ = vf.get_approximant("exp", "poly", 4, 0.0, 10.0)
    assert num[0] == pytest.approx(0.9666313, rel=1e-5)


def test_half_angle_polynomial(vf):
    """The exact angle's arctangent polynomial (VF_FN_HALF_ANGLE): the library's
    degree-7 fit of 2 atan(sqrt s) / sqrt s on [0, 1], so that A = u P(u^2)
    for u = tan(A/2) in [0, 1), reaches its minimax level (relative error
    about 1.1e-7 of the angle) and agrees with the oracle's independent Remez
    of the same function; the arctangent identity makes it exact on the
    closed forms A(0) = 0, A(u = tan(pi/8)) = pi/4, A(u = 1) = pi/2."""
    import math
    import numpy as np
    from oracle import remez as R
    num, den, eps = vf.get_approximant("half_angle", "poly", 7, 0.0, 1.0)
    assert den == [] and len(num) == 8
    assert eps < 2e-7
    P = np.polynomial.polynomial

    def g(s):
        s = np.asarray(s, dtype=np.float64)
        r = np.sqrt(np.maximum(s, 1e-300))
        return np.where(s > 0, 2 * np.arctan(r) / r, 2.0)

    ref = R.remez(g, 0.0, 1.0, 7)
    assert eps == pytest.approx(ref.eps, rel=1e-3)
    u = np.linspace(0.0, 1.0, 100001)
    ang = u * P.polyval(u * u, num)
    exact = 2 * np.arctan(u)
    rel = np.abs(ang - exact)[1:] / exact[1:]
    assert rel.max() <= 1.2e-7
    for uu, a in [(0.0, 0.0), (math.tan(math.pi / 8), math.pi / 4), (1.0, math.pi / 2)]:
        assert uu * P.polyval(uu * uu, num) == pytest.approx(a, rel=1.2e-7, abs=1e-12)
    with pytest.raises(vf.VFError):  # read-only
        vf.set_coefficients("half_angle", "poly", 7, num, lo=0.0, hi=1.0)


def test_alloc_failure_hook_without_gpu(vf):
    """vf_debug_fail_alloc: the countdown skips `after` allocations, fails the
    next one with VF_ERR_OOM (6) and disarms itself; a negative value
    disarms it.  vf_create's handle is a counted allocation."""
    L = vf.lib()
    ctx = ctypes.c_void_p()
    assert vf.debug_fail_alloc(0) == -1
    assert L.vf_create(ctypes.byref(ctx)) == 6 and not ctx.value
    assert vf.debug_fail_alloc(-1) == -1                   # it disarmed itself
    assert vf.debug_fail_alloc(1) == -1
    assert L.vf_create(ctypes.byref(ctx)) == 0 and ctx.value
    L.vf_destroy(ctx)
    ctx = ctypes.c_void_p()
    assert L.vf_create(ctypes.byref(ctx)) == 6 and not ctx.value
    assert vf.debug_fail_alloc(5) == -1
    assert vf.debug_fail_alloc(-7) == 5                    # disarmed before it fired
    assert L.vf_create(ctypes.byref(ctx)) == 0
    L.vf_destroy(ctx)
    assert vf.debug_fail_alloc(-1) == -1
