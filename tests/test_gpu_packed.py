"""Packed-precision (FP16x2 / BF16x2) pair terms with FP32 aggregation.

Bars, derived from the formats (unit roundoff 2^-11 for FP16, 2^-8 for BF16):
a packed distance or angle term carries a relative error of a few units of
roundoff, so an aggregate of n - 1 terms is within ~2 u relative of the exact
one: selections must equal the FP64 oracle's wherever the oracle's gap to the
best different colour exceeds 4e-3 (FP16) or 4e-2 (BF16).  The FP16 L1 term of
AMNF is exact (integers up to 765), so FP16 AMNF must equal the FP32 path byte
for byte.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import filters as F  # noqa: E402
from oracle import metrics as M  # noqa: E402
from paper_1009_0959_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

BAND = {"fp16x2": 4e-3, "bf16x2": 4e-2}


@pytest.fixture(scope="module")
def vf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0959_gb300 import build, vfilt
    build.build()
    return vfilt


def gpu(vf, img, **kw):
    t = torch.from_numpy(synth.to_rgbx(img)).cuda()
    out = vf.filter(t, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("w", [3, 5, 7])
@pytest.mark.parametrize("crit,approx", [("amnfe", "exact"), ("amnfe", "rational"),
                                         ("amnfg", "poly"), ("amnfg", "exact")])
def test_fp16_amnf_equals_fp32(vf, crit, approx, w):
    clean, noisy = synth.noisy(37, 131, 0.2, 40 + w)
    a = gpu(vf, noisy, criterion=crit, window=w, approx=approx, degree=4)
    b = gpu(vf, noisy, criterion=crit, window=w, approx=approx, degree=4, precision="fp16x2")
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp16x2", "bf16x2"])
@pytest.mark.parametrize("w", [3, 5, 7])
@pytest.mark.parametrize("crit,approx,deg", [("vmf", "exact", 4), ("bvdf", "poly", 4),
                                             ("bvdf", "poly", 2), ("evmf", "exact", 4),
                                             ("evmf", "rational", 4)])
def test_packed_selection_band(vf, crit, approx, deg, w, prec):
    """37 x 131: two 64-wide packed tiles and a ragged third, ragged rows."""
    clean, noisy = synth.noisy(37, 131, 0.2, 60 + w)
    o, d = F.filter_image(noisy, F.Config(crit, w, approx, deg))
    g = gpu(vf, noisy, criterion=crit, window=w, approx=approx, degree=deg, precision=prec)
    diff = np.any(o[..., :3] != g[..., :3], axis=-1)
    # the window's colours are the only possible outputs; EVMF's switch is
    # computed in FP32 and keeps the FP32 band
    safe = d["gap"] > BAND[prec]
    assert (diff & safe).sum() == 0, (diff & safe).sum()


@pytest.mark.parametrize("prec", ["fp16x2", "bf16x2"])
def test_packed_amnf_close(vf, prec):
    clean, noisy = synth.noisy(64, 96, 0.2, 7)
    o, _ = F.filter_image(noisy, F.Config("amnfe", 5, "rational", 4))
    g = gpu(vf, noisy, criterion="amnfe", window=5, approx="rational", precision=prec)
    err = np.abs(o[..., :3].astype(int) - g[..., :3].astype(int))
    assert err.max() <= (1 if prec == "fp16x2" else 8)


@pytest.mark.parametrize("shape", [(1, 1), (1, 70), (70, 1), (5, 130), (3, 65)])
@pytest.mark.parametrize("prec", ["fp16x2", "bf16x2"])
def test_packed_edge_shapes(vf, shape, prec):
    clean, noisy = synth.noisy(shape[0], shape[1], 0.3, 11)
    for crit, w in [("vmf", 7), ("evmf", 3)]:
        o, d = F.filter_image(noisy, F.Config(crit, w))
        g = gpu(vf, noisy, criterion=crit, window=w, precision=prec)
        diff = np.any(o[..., :3] != g[..., :3], axis=-1)
        assert (diff & (d["gap"] > BAND[prec])).sum() == 0
    o, _ = F.filter_image(noisy, F.Config("amnfg", 7))
    g = gpu(vf, noisy, criterion="amnfg", window=7, precision=prec)
    assert np.abs(o[..., :3].astype(int) - g[..., :3].astype(int)).max() <= 8


def test_packed_quality(vf):
    """Against the FP64 oracle's exact filter (256 x 256, 10 %): the FP16 VMF
    and the FP16 degree-4 BVDF change few selections and little PSNR."""
    clean, noisy = synth.noisy(256, 256, 0.10, 1)
    for crit, approx in [("vmf", "exact"), ("bvdf", "poly")]:
        ex, _ = F.filter_image(noisy, F.Config(crit, 3), threads=4)
        g = gpu(vf, noisy, criterion=crit, window=3, approx=approx, precision="fp16x2")
        assert M.changed_fraction(ex, g) <= 0.02
        assert M.psnr(clean, ex) - M.psnr(clean, g) <= 0.1


def test_packed_rejections(vf):
    t = torch.zeros((8, 8, 4), dtype=torch.uint8, device="cuda")
    o = torch.zeros_like(t)
    with pytest.raises(vf.VFError) as e:
        vf.filter(t, o, criterion="bvdf", approx="exact", precision="fp16x2")
    assert e.value.name == "VF_ERR_UNSUPPORTED"
    with pytest.raises(vf.VFError) as e:
        vf.Batch([(t, o, {"precision": "bf16x2"})])
    assert e.value.name == "VF_ERR_UNSUPPORTED"
