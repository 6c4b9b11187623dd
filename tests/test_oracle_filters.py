"""Pins of the oracle's filters (Sec. 3) against closed forms, library
routines on special cases, brute force and invariants.  CPU only."""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest
from scipy import ndimage

from oracle import filters as F
from oracle import metrics as M
from paper_1009_0959_gb300 import synth


def _grey(h, w, seed):
    v = synth.rand_int(seed, 99, np.arange(h * w), 0, 255).reshape(h, w).astype(np.uint8)
    return np.repeat(v[..., None], 3, axis=2), v


def _window(img, r, c, w):
    R = w // 2
    H, W = img.shape[:2]
    xs = []
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            xs.append(img[min(max(r + dy, 0), H - 1), min(max(c + dx, 0), W - 1), :3])
    return np.array(xs, dtype=np.float64)


# ---------------------------------------------------------------- VMF


@pytest.mark.parametrize("w", [3, 5, 7])
def test_vmf_grey_is_scalar_median(w):
    """On grey images ||x_i - x_j||_2 = sqrt(3)|v_i - v_j|, so the VMF output is
    the scalar median of the window: scipy's median filter, borders 'nearest'
    (the clamp-to-edge reading)."""
    img, v = _grey(23, 31, 7 + w)
    out, _ = F.filter_image(img, F.Config("vmf", w))
    ref = ndimage.median_filter(v, size=w, mode="nearest")
    np.testing.assert_array_equal(out[..., 0], ref)
    np.testing.assert_array_equal(out[..., 1], ref)


def test_vmf_brute_force_decimal():
    """Aggregates of tiny random windows against 40-digit decimal arithmetic."""
    getcontext().prec = 40
    rng = np.random.default_rng(3)
    cfg = F.Config("vmf", 3)
    for _ in range(20):
        xs = rng.integers(0, 256, size=(9, 3)).astype(np.float64)
        agg = F.window_aggregates(cfg, xs)
        for i in range(9):
            s = Decimal(0)
            for j in range(9):
                d2 = sum(int(xs[i, k] - xs[j, k]) ** 2 for k in range(3))
                s += Decimal(d2).sqrt()
            assert abs(float(s) - agg[i]) <= 1e-12 * max(1.0, float(s))


def test_vmf_permutation_invariance():
    rng = np.random.default_rng(4)
    cfg = F.Config("vmf", 5)
    xs = rng.integers(0, 256, size=(25, 3)).astype(np.float64)
    agg = F.window_aggregates(cfg, xs)
    perm = rng.permutation(25)
    np.testing.assert_allclose(F.window_aggregates(cfg, xs[perm]), agg[perm], rtol=1e-13)


@pytest.mark.parametrize("crit", ["vmf", "bvdf", "evmf"])
def test_selection_output_in_window(crit):
    clean, noisy = synth.noisy(40, 37, 0.2, 11)
    out, d = F.filter_image(noisy, F.Config(crit, 3))
    for r in range(0, 40, 3):
        for c in range(0, 37, 3):
            win = _window(noisy, r, c, 3)
            assert (win == out[r, c, :3]).all(axis=1).any()
            np.testing.assert_array_equal(win[d["sel"][r, c]], out[r, c, :3])


@pytest.mark.parametrize("crit", ["vmf", "bvdf", "amnfe", "amnfg", "evmf"])
@pytest.mark.parametrize("approx", ["exact", "poly"])
def test_constant_image_unchanged(crit, approx):
    img = np.zeros((9, 11, 3), np.uint8)
    img[...] = (200, 120, 40)
    out, _ = F.filter_image(img, F.Config(crit, 5, approx, 4))
    np.testing.assert_array_equal(out, img)


@pytest.mark.parametrize("crit", ["vmf", "bvdf", "amnfe", "evmf"])
def test_impulse_removed(crit):
    """An isolated impulse of another direction in a flat window is removed
    (AMNF: pulled to within one level of the flat value)."""
    img = np.zeros((7, 7, 3), np.uint8)
    img[...] = (90, 140, 60)
    img[3, 3] = (250, 10, 200)
    out, _ = F.filter_image(img, F.Config(crit, 3))
    if crit == "amnfe":
        assert np.abs(out[3, 3].astype(int) - (90, 140, 60)).max() <= 1
    else:
        np.testing.assert_array_equal(out[3, 3], (90, 140, 60))


@pytest.mark.parametrize("crit", ["vmf", "bvdf", "evmf", "evbdf", "amnfe", "amnfg"])
def test_fourth_byte_convention(crit):
    """RGBX images: only the first three bytes are colour (Sec. 3: RGB
    vectors).  The library's convention for the fourth byte: a selection
    (VMF, BVDF, the switched EVMF / EVBDF, or their centre when not switched)
    carries the selected sample's pixel's byte, a weighted mean (AMNF) the
    centre pixel's.  Checked on random fourth bytes, borders included."""
    clean, noisy = synth.noisy(13, 17, 0.3, 44)
    rng = np.random.default_rng(45)
    img = np.concatenate([noisy, rng.integers(0, 256, (13, 17, 1)).astype(np.uint8)], axis=2)
    out, d = F.filter_image(img, F.Config(crit, 3))
    np.testing.assert_array_equal(out[..., :3], F.filter_image(noisy, F.Config(crit, 3))[0])
    for r in range(13):
        for c in range(17):
            s = d["sel"][r, c]
            if s < 0:
                src = (r, c)
            else:
                src = (min(max(r + s // 3 - 1, 0), 12), min(max(c + s % 3 - 1, 0), 16))
                assert (img[src][:3] == out[r, c, :3]).all()
            assert out[r, c, 3] == img[src][3]
    assert (d["sel"] >= 0).any() if crit not in ("amnfe", "amnfg") else (d["sel"] < 0).all()


def test_border_replicates():
    """1 x 1 and 1 x n images: every window repeats border pixels."""
    img = np.array([[[10, 20, 30]]], np.uint8)
    for crit in ["vmf", "bvdf", "amnfe", "evmf"]:
        out, _ = F.filter_image(img, F.Config(crit, 7))
        np.testing.assert_array_equal(out, img)
    row = np.array([[[0, 0, 0], [100, 100, 100], [0, 0, 0]]], np.uint8)
    out, _ = F.filter_image(row, F.Config("vmf", 3))
    # centre window: columns (0,1,2) x 3 replicated rows: six zeros, three 100s
    np.testing.assert_array_equal(out[0, 1], (0, 0, 0))


# ---------------------------------------------------------------- BVDF


def test_angle_known_values():
    for a, b, ang in [((1, 0, 0), (0, 1, 0), math.pi / 2), ((1, 1, 0), (1, 0, 0), math.pi / 4),
                      ((3, 6, 9), (1, 2, 3), 0.0), ((0, 0, 0), (5, 1, 2), math.pi / 2),
                      ((1, 1, 1), (1, 0, 0), math.acos(1 / math.sqrt(3)))]:
        assert F.angle(a, b) == pytest.approx(ang, abs=1e-15)


def test_angle_exact_matches_acos_form():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        a, b = rng.integers(0, 256, 3), rng.integers(0, 256, 3)
        e, c = F.angle(a, b), F.angle(a, b, "acos")
        # arccos of a rounded cosine loses up to sqrt(eps) near 0
        assert abs(e - c) <= 3e-8


@pytest.mark.parametrize("degree", [2, 4, 6])
def test_angle_approx_within_eps(degree):
    """The piecewise approximant stays within the larger of the two pieces'
    minimax errors of the exact angle, on both sides of z = 0.5."""
    from oracle import approximants as AP
    cfg = F.Config("bvdf", 3, "poly", degree)
    eps = max(AP.fit("acos_lo", degree, *AP.ACOS_LO_INTERVAL).eps,
              AP.fit("acos_hi", degree, *AP.ACOS_HI_INTERVAL).eps)
    rng = np.random.default_rng(6)
    worst, seen_lo, seen_hi = 0.0, 0, 0
    for _ in range(3000):
        a, b = rng.integers(1, 256, 3), rng.integers(1, 256, 3)
        z = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        seen_lo += z < 0.5
        seen_hi += z >= 0.5
        worst = max(worst, abs(F.angle(a, b, "approx", cfg) - F.angle(a, b)))
    assert seen_lo > 10 and seen_hi > 10
    assert worst <= eps * (1 + 1e-6) + 1e-12


def test_bvdf_grey_ties_to_lowest_index():
    """On a grey image all angles are 0: every aggregate ties and the lowest
    raster index (the top-left sample) is selected, i.e. the image shifts by
    one pixel down-right with replicated borders."""
    img, v = _grey(9, 12, 8)
    img[img == 0] = 1  # keep the cosine defined
    out, d = F.filter_image(img, F.Config("bvdf", 3))
    assert (d["sel"] == 0).all()
    ref = img[np.clip(np.arange(9) - 1, 0, 8)][:, np.clip(np.arange(12) - 1, 0, 11)]
    np.testing.assert_array_equal(out, ref)


def test_bvdf_scaled_impulse_kept():
    """An impulse that is a multiple of the flat colour has angle 0 to every
    sample: BVDF sees no outlier (the lowest index is chosen, which is a flat
    sample, so the output is still the flat colour); an impulse of another
    direction loses."""
    img = np.zeros((5, 5, 3), np.uint8)
    img[...] = (40, 60, 80)
    img[2, 2] = (80, 120, 160)
    cfg = F.Config("bvdf", 3)
    xs = _window(img, 2, 2, 3)
    agg = F.window_aggregates(cfg, xs)
    np.testing.assert_allclose(agg, 0.0, atol=1e-12)


def test_bvdf_sums_angles_not_cosine_distances():
    """BVDF ranks each sample by the sum of its angles to the others (Sec.
    3.1).  A 3 x 3 window in the R-G plane: five samples along R (0 deg), one
    at theta = atan(100/173), about 30 deg, three along G (90 deg).  Angle
    sums: R theta + 3 pi/2 (about 300 deg), the middle sample 5 theta +
    3 (pi/2 - theta) (about 330 deg), G 5 pi/2 + pi/2 - theta (about 510
    deg), so an R sample wins, the first in raster order.  Summing the
    cosine distance 1 - cos instead (3.13, 2.17, 5.50) would pick the
    middle sample."""
    r, m, g = (200, 0, 0), (173, 100, 0), (0, 200, 0)
    img = np.array([[r, r, g], [r, m, r], [g, r, g]], np.uint8)
    th = math.atan2(100, 173)
    want = {r: th + 3 * math.pi / 2, m: 5 * th + 3 * (math.pi / 2 - th),
            g: 5 * math.pi / 2 + (math.pi / 2 - th)}
    xs = _window(img, 1, 1, 3)
    agg = F.window_aggregates(F.Config("bvdf", 3), xs)
    for x, v in zip(xs, agg):
        assert v == pytest.approx(want[tuple(int(t) for t in x)], rel=1e-12)
    out, d = F.filter_image(img, F.Config("bvdf", 3))
    assert d["sel"][1, 1] == 0
    assert tuple(out[1, 1]) == r


# ---------------------------------------------------------------- AMNF


@pytest.mark.parametrize("crit", ["amnfe", "amnfg"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_amnf_two_value_closed_form(crit, k):
    """Window of n - k samples equal to a (incl. the centre) and k equal to b,
    d1 = ||a - b||_1, d2 = ||a - b||_2.  Then h_a = n^(-kappa/3) k d1,
    h_b = n^(-kappa/3) (n - k) d1, the a-weights are h_a^-3 K(0) = h_a^-3 and
    the b-weights h_b^-3 K((a - b)/h_b), so y is a two-point mean."""
    n, kappa = 9, 0.33
    a = np.array([100.0, 120.0, 90.0])
    b = np.array([160.0, 30.0, 200.0])
    xs = np.tile(a, (n, 1))
    xs[[0, 2, 8][:k]] = b
    d1, d2 = np.abs(a - b).sum(), np.sqrt(((a - b) ** 2).sum())
    s = n ** (-kappa / 3)
    ha, hb = s * k * d1, s * (n - k) * d1
    kb = math.exp(-d1 / hb) if crit == "amnfe" else math.exp(-0.5 * (d2 / hb) ** 2)
    wa, wb = ha ** -3, hb ** -3 * kb
    y = ((n - k) * wa * a + k * wb * b) / ((n - k) * wa + k * wb)
    got = F.window_amnf(F.Config(crit, 3), xs)
    np.testing.assert_allclose(got, y, rtol=1e-13)
    # the filter writes y rounded to the nearest 8-bit level (the output is a
    # colour of the 8-bit image): the same window as a 3 x 3 image, centre
    # output; y has no channel near a half level, and channels with a
    # fraction above one half tell rounding from truncation
    frac = y - np.floor(y)
    assert (np.abs(frac - 0.5) > 1e-6).all()
    out, _ = F.filter_image(xs.reshape(3, 3, 3).astype(np.uint8), F.Config(crit, 3))
    np.testing.assert_array_equal(out[1, 1], np.floor(y) + (frac > 0.5))


def test_amnf_within_window_range():
    clean, noisy = synth.noisy(30, 30, 0.3, 12)
    for crit in ["amnfe", "amnfg"]:
        _, d = F.filter_image(noisy, F.Config(crit, 3))
        y = d["yreal"]
        for r in range(30):
            for c in range(30):
                win = _window(noisy, r, c, 3)
                assert (y[r, c] >= win.min(0) - 1e-9).all()
                assert (y[r, c] <= win.max(0) + 1e-9).all()


def test_amnf_argument_bound():
    """d1_Ci <= sum_j d1_ij, so z = d1_Ci / h_i <= n^(kappa/3): the EXP
    argument never reaches the cut-off 10.  Checked through the cut-off: a
    cut-off just above the bound leaves the exact output unchanged."""
    clean, noisy = synth.noisy(24, 24, 0.3, 13)
    for w in (3, 5):
        n = w * w
        ref, _ = F.filter_image(noisy, F.Config("amnfe", w))
        cut, _ = F.filter_image(noisy, F.Config("amnfe", w, exp_cutoff=n ** (0.33 / 3) + 1e-9))
        np.testing.assert_array_equal(ref, cut)


def test_exp_at_zero_and_cutoff():
    cfg = F.Config("amnfe", 3)
    assert F.expneg(cfg, 0.0) == 1.0
    assert F.expneg(cfg, 10.5) == 0.0
    capx = F.Config("amnfe", 3, "rational")
    assert F.expneg(capx, 10.5) == 0.0


# ---------------------------------------------------------------- EVMF


def test_evmf_switch_closed_form():
    """With no cut-off, P_C > beta_C <=> P_C > exp(-H), H = -sum_j P_j ln P_j
    (divide the inequality by P_C > 0 and take logs)."""
    rng = np.random.default_rng(9)
    cfg = F.Config("evmf", 3, ent_cutoff=0.0)
    agree = 0
    for _ in range(3000):
        xs = rng.integers(0, 256, size=(9, 3)).astype(np.float64)
        if rng.random() < 0.5:  # flatter windows with one outlier
            xs[:] = xs[0] + rng.integers(-6, 7, size=(9, 3))
            xs[rng.integers(9)] = rng.integers(0, 256, 3)
        xs = np.clip(xs, 0, 255)
        mean = xs.mean(0)
        r = np.sqrt(((xs - mean) ** 2).sum(1))
        P = r / r.sum()
        H = -sum(p * math.log(p) for p in P if p > 0)
        expect = P[4] > math.exp(-H)
        got, gap = F.window_evmf_switch(cfg, xs)
        if gap > 1e-9:
            assert got == expect
            agree += 1
    assert agree > 2900


@pytest.mark.parametrize("w", [3, 5, 7])
def test_evmf_worked_example(w):
    """Flat window with a centre impulse: P_C = 1/2, P_i = 1/(2(n-1)),
    exp(-H) = 1/(2 sqrt(n-1)) < 1/2, so the filter switches and outputs the
    flat colour (the vector median)."""
    n = w * w
    xs = np.tile([50.0, 80.0, 120.0], (n, 1))
    xs[n // 2] = [250.0, 10.0, 30.0]
    mean = xs.mean(0)
    r = np.sqrt(((xs - mean) ** 2).sum(1))
    assert r[n // 2] / r.sum() == pytest.approx(0.5, rel=1e-14)
    sw, _ = F.window_evmf_switch(F.Config("evmf", w, ent_cutoff=0.0), xs)
    assert sw
    img = xs.reshape(w, w, 3).astype(np.uint8)
    out, d = F.filter_image(img, F.Config("evmf", w, ent_cutoff=0.0))
    assert d["sw"][w // 2, w // 2] == 1
    np.testing.assert_array_equal(out[w // 2, w // 2], (50, 80, 120))


def test_evmf_flat_identity():
    img = np.zeros((6, 6, 3), np.uint8)
    img[...] = (1, 2, 3)
    out, d = F.filter_image(img, F.Config("evmf", 3))
    assert d["sw"].sum() == 0
    np.testing.assert_array_equal(out, img)


def test_evmf_cutoff_reading():
    """With the cut-off, ENT(P_C) = 0 whenever P_C < T, so beta_C = 0 and the
    filtering branch is taken (the behaviour of the paper's cut-off read as
    part of ENT)."""
    xs = np.tile([100.0, 100.0, 100.0], (9, 1))
    xs[:, 0] += [-9, 5, 9, -7, 1, 7, -5, 3, -4]  # P_C = 1/50 < 0.05
    sw_cut, _ = F.window_evmf_switch(F.Config("evmf", 3), xs)
    sw_plain, _ = F.window_evmf_switch(F.Config("evmf", 3, ent_cutoff=0.0), xs)
    assert sw_cut and not sw_plain


def test_evmf_cutoff_tie_reported():
    """A P_j exactly at the ENT cut-off T = 1/20 (Sec. 3.3) is a threshold
    decision that rounding may take either way: the diagnostic gap reports it
    as a near tie.  Blue channel {131, 166 x 6, 236 x 2} (R, G fixed): mean
    1599/9, distances 420/9, 105/9 and 525/9, sum 2100/9, so P = 105/2100 =
    1/20 for the six 166s.  With 130 instead of 131 the sum is 2104/9 and
    P = 104/2104: gap 1 - 20 * 104 / 2104 = 24/2104."""
    def win(b0):
        img = np.zeros((3, 3, 3), np.uint8)
        img[..., 0], img[..., 1] = 173, 169
        img[..., 2] = np.array([[b0, 166, 166], [166, 236, 166], [166, 236, 166]])
        return img
    _, d = F.filter_image(win(131), F.Config("evmf", 3))
    assert d["gap"][1, 1] < 1e-12
    _, d = F.filter_image(win(130), F.Config("evmf", 3))
    assert d["gap"][1, 1] == pytest.approx(24 / 2104, rel=1e-12)
    _, d = F.filter_image(win(131), F.Config("evmf", 3, ent_cutoff=0.0))
    assert d["gap"][1, 1] > 0.1  # no cut-off: only the switch's own gap


@pytest.mark.parametrize("crit", ["amnfe", "amnfg"])
def test_amnf_cutoff_tie_reported(crit):
    """An argument of E exactly at the EXP cut-off (Sec. 3.2) is reported as a
    near tie: with the cut-off set to sample k's argument z_k =
    ||(x_C - x_k) / h_k|| (L1 for AMNFE, half the squared L2 for AMNFG; h_k =
    n^(-kappa/3) sum_j ||x_k - x_j||_1), the centre's gap is 0 up to rounding."""
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, (3, 3, 3)).astype(np.uint8)
    x = img.reshape(9, 3).astype(np.float64)
    h = 9.0 ** (-0.33 / 3.0) * np.abs(x[:, None, :] - x[None, :, :]).sum(-1).sum(1)
    dc = x[4] - x
    z = np.abs(dc).sum(1) / h if crit == "amnfe" else 0.5 * (dc ** 2).sum(1) / h ** 2
    k = int(np.argmax(z))
    _, d = F.filter_image(img, F.Config(crit, 3, exp_cutoff=float(z[k])))
    assert d["gap"][1, 1] < 1e-12
    _, d = F.filter_image(img, F.Config(crit, 3))
    y = d["yreal"][1, 1]
    assert d["gap"][1, 1] == pytest.approx(np.abs(y - np.floor(y) - 0.5).min(), rel=1e-9)


def test_ent_values():
    cfg = F.Config("evmf", 3)
    assert F.ent(cfg, 0.04) == 0.0
    assert F.ent(cfg, 0.5) == pytest.approx(0.5 * math.log(0.5), rel=1e-15)
    assert F.ent(F.Config("evmf", 3, ent_cutoff=0.0), 0.0) == 0.0


# ---------------------------------------------------------------- noise, metrics


def test_noise_rates():
    clean = synth.piecewise_smooth(200, 200, 21)
    n = clean.size
    for p in (0.05, 0.3):
        noisy = synth.impulse_uncorrelated(clean, p, 21)
        # a replaced channel equals the old value with probability 1/256
        rate = (noisy != clean).mean() / (1 - 1 / 256)
        assert abs(rate - p) < 4 * math.sqrt(p * (1 - p) / n)
    noisy = synth.impulse_correlated(clean, 0.4, 22)
    changed = noisy != clean
    px = changed.any(-1)
    frac = px.mean() / (1 - (1 / 256))
    assert abs(frac - 0.4) < 0.01
    pats = changed[px].astype(int) @ np.array([1, 2, 4])
    counts = np.array([(pats == v).mean() for v in (1, 2, 4)])
    assert np.all(np.abs(counts - 0.25) < 0.02)
    assert (pats == 7).mean() > 0.2


def test_impulse_values_uniform():
    """Eq. eq_noise: a replaced channel takes a random value r_k, uniform on
    0..255 (random-valued impulses, not salt-and-pepper): over 95,000-115,000
    replaced channels of a flat image every level occurs, with mean 127.5 and
    standard deviation sqrt((256^2 - 1) / 12) = 73.9 within sampling error."""
    flat = np.full((400, 400, 3), 77, np.uint8)
    for noisy in (synth.impulse_uncorrelated(flat, 0.24, 31),
                  synth.impulse_correlated(flat, 0.4, 32)):
        v = noisy[noisy != 77].astype(np.float64)
        assert v.size > 90_000
        assert len(np.unique(v)) == 255  # every level but the flat one
        sd = math.sqrt((256 ** 2 - 1) / 12.0)
        assert abs(v.mean() - 127.5) < 4 * sd / math.sqrt(v.size) + 0.3
        assert v.std() == pytest.approx(sd, rel=0.01)


def test_gaussian_noise_sigma():
    """The Gaussian part of the mixed model: zero mean, standard deviation
    sigma (here 10 levels on a flat mid-grey image, far from the clamps)."""
    flat = np.full((300, 300, 3), 128, np.uint8)
    d = synth.gaussian(flat, 10.0, 41).astype(np.float64) - 128.0
    assert abs(d.mean()) < 4 * 10.0 / math.sqrt(d.size)
    # rounding to integers adds variance 1/12
    assert d.std() == pytest.approx(math.sqrt(100.0 + 1.0 / 12.0), rel=0.01)


def test_generator_deterministic():
    a = synth.noisy(64, 48, 0.1, 5)[1]
    b = synth.noisy(64, 48, 0.1, 5)[1]
    np.testing.assert_array_equal(a, b)
    c = synth.noisy(64, 48, 0.1, 6)[1]
    assert (a != c).any()


def test_generator_channel_correlation():
    img = synth.piecewise_smooth(256, 256, 1).reshape(-1, 3).astype(float)
    cc = np.corrcoef(img.T)
    assert cc[np.triu_indices(3, 1)].mean() > 0.7


def test_metrics():
    a = synth.piecewise_smooth(32, 32, 3)
    assert M.mae(a, a) == 0.0 and M.mse(a, a) == 0.0 and M.ncd(a, a) == 0.0
    b = a.astype(int)
    b[..., 0] = np.clip(b[..., 0] + 0, 0, 255)
    lab_white = M.srgb_to_lab(np.array([[255, 255, 255]], np.uint8))[0]
    np.testing.assert_allclose(lab_white, [100.0, 0.0, 0.0], atol=1e-9)
    red = M.srgb_to_lab(np.array([[255, 0, 0]], np.uint8))[0]
    np.testing.assert_allclose(red, [53.24, 80.09, 67.20], atol=0.1)  # textbook sRGB red
    # a mid-tone exercises the sRGB transfer curve: sRGB (128, 128, 128) is
    # L* 53.59, a* = b* = 0 in the standard conversion tables
    grey = M.srgb_to_lab(np.array([[128, 128, 128]], np.uint8))[0]
    np.testing.assert_allclose(grey, [53.59, 0.0, 0.0], atol=0.01)
    # NCD: summed Lab distances over summed Lab norms of the first image;
    # white vs red per pixel |(100, 0, 0) - (53.24, 80.09, 67.20)| / 100
    wr = math.sqrt(46.76 ** 2 + 80.09 ** 2 + 67.20 ** 2) / 100.0
    white = np.full((1, 2, 3), 255, np.uint8)
    both_red = np.array([[[255, 0, 0], [255, 0, 0]]], np.uint8)
    one_red = np.array([[[255, 255, 255], [255, 0, 0]]], np.uint8)
    assert M.ncd(white, both_red) == pytest.approx(wr, rel=2e-3)
    assert M.ncd(white, one_red) == pytest.approx(wr / 2, rel=2e-3)
    c = np.full((10, 10, 3), 100, np.uint8)
    d = c + 2
    assert M.psnr(c, d) == pytest.approx(10 * math.log10(255 ** 2 / 4))
    assert M.mae(c, d) == pytest.approx(2.0)


# ---------------------------------------------------------------- generalised EVF (EVBDF)


@pytest.mark.parametrize("w", [3, 5])
@pytest.mark.parametrize("approx,deg", [("exact", 4), ("poly", 4)])
def test_evbdf_is_switch_then_bvdf(w, approx, deg):
    """Sec. 3.3 generalised EVF with the angle of Sec. 3.1 in the filtering
    branch: wherever EVMF's switch fires the output is BVDF's, elsewhere the
    centre; the switch is EVMF's own (same ENT approximant)."""
    clean, noisy = synth.noisy(30, 41, 0.2, 31 + w)
    o_ev, d_ev = F.filter_image(noisy, F.Config("evbdf", w, approx, deg))
    o_em, d_em = F.filter_image(noisy, F.Config("evmf", w, approx, deg))
    o_bv, _ = F.filter_image(noisy, F.Config("bvdf", w, approx, deg))
    np.testing.assert_array_equal(d_ev["sw"], d_em["sw"])
    sw = d_ev["sw"].astype(bool)
    assert 0 < sw.mean() < 1
    np.testing.assert_array_equal(o_ev[sw], o_bv[sw])
    np.testing.assert_array_equal(o_ev[~sw], noisy[~sw])


@pytest.mark.parametrize("w", [3, 5])
def test_evbdf_worked_example(w):
    """Flat window with a centre impulse of another direction: switched (as
    for EVMF), and the angular selection returns the flat colour; with an
    impulse parallel to the flat colour the angles cannot tell them apart
    (all zero): the lowest index, a flat sample, again."""
    n = w * w
    for imp in ([250.0, 10.0, 30.0], [100.0, 160.0, 240.0]):  # other direction; 2x flat
        xs = np.tile([50.0, 80.0, 120.0], (n, 1))
        xs[n // 2] = imp
        img = xs.reshape(w, w, 3).astype(np.uint8)
        out, d = F.filter_image(img, F.Config("evbdf", w, ent_cutoff=0.0))
        assert d["sw"][w // 2, w // 2] == 1
        np.testing.assert_array_equal(out[w // 2, w // 2], (50, 80, 120))
