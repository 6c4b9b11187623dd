"""The fourth byte of RGBX images.  Only the first three bytes are colour
(Sec. 3: RGB vectors); the library's convention is that a selection carries
the selected sample's pixel's fourth byte and a weighted mean (AMNF) the
centre pixel's.  Where several samples of the window share the selected
colour, any of them is a valid selection (their aggregates are equal in exact
arithmetic, and FP32 may order them either way), so the check accepts the
fourth byte of any of them.

`fourth_byte_valid` is checked on the CPU against the oracle (which follows
the convention) and against planted mistakes; the `-m gpu` cases run it on
the library's output for random fourth bytes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import filters as F  # noqa: E402
from paper_1009_0959_gb300 import synth  # noqa: E402


def fourth_byte_valid(img, out, window, crit):
    """Per pixel: AMNF -- the centre's fourth byte; a selection -- the
    output colour is a window sample's (borders replicated), and its fourth
    byte is that of a window sample of that colour.  Returns the number of
    pixels that break the convention."""
    H, W, _ = img.shape
    R = window // 2
    pad = np.pad(img, ((R, R), (R, R), (0, 0)), mode="edge")
    if crit in ("amnfe", "amnfg"):
        return int((out[..., 3] != img[..., 3]).sum())
    ok = np.zeros((H, W), bool)
    colour_found = np.zeros((H, W), bool)
    for dy in range(window):
        for dx in range(window):
            s = pad[dy:dy + H, dx:dx + W]
            same = np.all(s[..., :3] == out[..., :3], axis=-1)
            colour_found |= same
            ok |= same & (s[..., 3] == out[..., 3])
    return int((~(ok & colour_found)).sum())


def _rgbx(h, w, seed):
    clean, noisy = synth.noisy(h, w, 0.25, seed)
    rng = np.random.default_rng(seed + 1)
    x = rng.integers(0, 256, (h, w, 1)).astype(np.uint8)
    return np.ascontiguousarray(np.concatenate([noisy, x], axis=2))


CRITS = [("vmf", "exact", 4), ("bvdf", "exact", 4), ("bvdf", "poly", 4), ("evmf", "exact", 4),
         ("evbdf", "poly", 4), ("amnfe", "exact", 4), ("amnfg", "rational", 4)]


@pytest.mark.parametrize("crit,approx,deg", CRITS)
def test_checker_accepts_the_oracle_and_catches_mistakes(crit, approx, deg):
    img = _rgbx(21, 29, 60)
    out, _ = F.filter_image(img, F.Config(crit, 5, approx, deg))
    assert fourth_byte_valid(img, out, 5, crit) == 0
    bad = out.copy()
    bad[..., 3] ^= 0x5A  # fourth bytes from nowhere
    assert fourth_byte_valid(img, bad, 5, crit) > 0
    if crit not in ("amnfe", "amnfg"):
        # the centre's byte where another sample was selected (a plausible slip)
        wrong = out.copy()
        wrong[..., 3] = img[..., 3]
        changed = np.any(out[..., :3] != img[..., :3], axis=-1)
        assert changed.any()
        assert fourth_byte_valid(img, wrong, 5, crit) > 0


@pytest.fixture(scope="module")
def vf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0959_gb300 import build, vfilt
    build.build()
    return vfilt


@pytest.mark.gpu
@pytest.mark.parametrize("reuse", [0, 1, 2])
@pytest.mark.parametrize("window", [3, 5, 7])
@pytest.mark.parametrize("crit,approx,deg", CRITS)
def test_gpu_fourth_byte(vf, crit, approx, deg, window, reuse):
    img = _rgbx(37, 67, 70 + window)
    t = torch.from_numpy(img).cuda()
    try:
        vf.set_option("pair_reuse", reuse)
        out = vf.filter(t, criterion=crit, window=window, approx=approx, degree=deg)
        torch.cuda.synchronize()
    finally:
        vf.set_option("pair_reuse", 1)
    assert fourth_byte_valid(img, out.cpu().numpy(), window, crit) == 0
