"""Parity at the full sizes of the precision, batched and gated workloads, in
the launch configuration the benchmark times, on sampled rows the FP64 oracle
computes one by one (top and bottom borders, the middle):

* one 4096 x 4096 image at 20 % impulses (seed 8), 5 x 5 and 7 x 7 windows:
  FP32 criteria (with the library's own rationals) with the single-image
  bar, FP16x2 and BF16x2 with their selection bands;
* the 256-image batch (320x240 .. 1920x1080, seed 9, windows 3/5/7 and the
  five criteria round-robin), autotuned and replayed as a CUDA graph: a
  sample of images, three row bands each;
* one 3840 x 2160 video frame through the gated filter (flags: the
  generator's impulse mask; the gate's own inference run at the same size):
  flagged pixels meet the oracle's bar on sampled rows, the others are the
  input unchanged.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import filters as F  # noqa: E402
from paper_1009_0959_gb300 import synth  # noqa: E402

from test_gpu_parity import check  # noqa: E402

pytestmark = pytest.mark.gpu

# the packed formats' selection bands (relative aggregate gap)
BAND = {"fp16x2": 4e-3, "bf16x2": 4e-2}


@pytest.fixture(scope="module")
def vf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0959_gb300 import build, vfilt
    build.build()
    return vfilt


def bands(h, k=3):
    """Row ranges: the first and last k rows (borders) and k in the middle."""
    m = h // 2
    return [(0, k), (m - 1, m - 1 + k), (h - k, h)]


def check_rows(crit, noisy, cfg, out, rows):
    for r0, r1 in rows:
        o, d = F.filter_image(noisy, cfg, rows=(r0, r1))
        sl = slice(r0, r1)
        check(crit, o[sl], {k: v[sl] for k, v in d.items()}, out[sl])


@pytest.fixture(scope="module")
def big(vf):
    clean, noisy = synth.noisy(4096, 4096, 0.20, 8)
    return noisy, torch.from_numpy(synth.to_rgbx(noisy)).cuda()


@pytest.mark.parametrize("w", [5, 7])
@pytest.mark.parametrize("crit,approx,deg", [("vmf", "exact", 4), ("bvdf", "exact", 4),
                                             ("bvdf", "poly", 4), ("amnfe", "rational", 4),
                                             ("amnfg", "poly", 4), ("evmf", "poly", 4),
                                             ("evbdf", "poly", 4), ("amnfe", "rational_fit", 3),
                                             ("evmf", "rational_fit", 4)])
def test_4096_fp32_sampled(vf, big, crit, approx, deg, w):
    noisy, t = big
    out = vf.filter(t, criterion=crit, window=w, approx=approx, degree=deg)
    torch.cuda.synchronize()
    check_rows(crit, noisy, F.Config(crit, w, approx, deg), out.cpu().numpy(), bands(4096))


@pytest.mark.parametrize("prec", ["fp16x2", "bf16x2"])
@pytest.mark.parametrize("w", [5, 7])
@pytest.mark.parametrize("crit,approx", [("vmf", "exact"), ("bvdf", "poly"), ("evmf", "poly")])
def test_4096_packed_sampled(vf, big, crit, approx, w, prec):
    noisy, t = big
    out = vf.filter(t, criterion=crit, window=w, approx=approx, degree=4,
                    precision=prec).cpu().numpy()
    for r0, r1 in bands(4096):
        o, d = F.filter_image(noisy, F.Config(crit, w, approx, 4), rows=(r0, r1))
        sl = slice(r0, r1)
        diff = np.any(o[sl, :, :3] != out[sl, :, :3], axis=-1)
        assert (diff & (d["gap"][sl] > BAND[prec])).sum() == 0


BATCH_CRITS = ["vmf", "bvdf", "amnfe", "amnfg", "evmf"]
BATCH_MINIMAX = {"vmf": ("exact", 4), "bvdf": ("poly", 4), "amnfe": ("rational", 4),
                 "amnfg": ("poly", 3), "evmf": ("poly", 5)}


def test_batch_256_sampled(vf):
    items = synth.batch_images(256, 9)
    dev = []
    for i, (clean, noisy, p) in enumerate(items):
        crit = BATCH_CRITS[i % 5]
        approx, deg = ("exact", 4) if (i // 15) % 2 == 0 else BATCH_MINIMAX[crit]
        params = dict(criterion=crit, window=(3, 5, 7)[i % 3], approx=approx, degree=deg)
        t = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
        dev.append((t, torch.zeros_like(t), params))
    b = vf.Batch(dev)
    b.autotune()
    for _, o, _ in dev:
        o.zero_()
    b.graph_launch()
    torch.cuda.synchronize()
    # every 8th image plus the first 15 (one of each criterion x window)
    for i in sorted(set(range(15)) | set(range(0, 256, 8))):
        noisy = items[i][1]
        p = dev[i][2]
        out = dev[i][1].cpu().numpy()
        cfg = F.Config(p["criterion"], p["window"], p["approx"], p["degree"])
        check_rows(p["criterion"], noisy, cfg, out, bands(noisy.shape[0], 2))
    b.close()


def test_gated_frame_3840x2160(vf):
    clean, noisy, p = synth.video_frame(2160, 3840, 40, 64, 265)
    t = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
    gate = vf.Gate(265)
    probe = gate.infer(t, 0.5)  # the gate's inference at this size: one flag per pixel
    torch.cuda.synchronize()
    assert probe.shape == (2160, 3840) and int(probe.max().item()) <= 1
    gate.close()
    # the flags a trained gate approximates: the generator's impulse mask
    mask = synth.impulse_mask(clean, noisy)
    flags = torch.from_numpy(mask.astype(np.uint8)).cuda()
    kw = dict(criterion="bvdf", window=5, approx="poly", degree=4)
    gated = vf.filter_gated(t, flags, **kw)
    torch.cuda.synchronize()
    m = flags.bool().unsqueeze(-1).expand_as(t)
    assert torch.equal(gated[~m], t[~m])  # unflagged pixels untouched
    g = gated.cpu().numpy()
    for r0, r1 in bands(2160):
        o, d = F.filter_image(noisy, F.Config("bvdf", 5, "poly", 4), rows=(r0, r1))
        sl = slice(r0, r1)
        diff = np.any(o[sl, :, :3] != g[sl, :, :3], axis=-1)
        assert (diff & mask[sl] & (d["gap"][sl] > 1e-5)).sum() == 0


@pytest.mark.parametrize("crit,w,approx", [("vmf", 5, "exact"), ("bvdf", 5, "poly"),
                                           ("evmf", 5, "poly"), ("amnfe", 7, "rational")])
def test_image_over_4gib(vf, crit, w, approx):
    """A 40000 x 32768 RGBX image (5.2 GB in, 5.2 GB out: byte offsets past
    2^32) made on the device by tiling a 512 x 512 synthetic tile; the rows
    at the top and bottom borders and the rows around the 4 GiB offset meet
    the oracle's bar (the oracle sees those rows with their vertical halo and
    the full width)."""
    H, W = 40000, 32768
    free, _ = torch.cuda.mem_get_info()
    if free < 16 * 2 ** 30:
        pytest.skip("needs 16 GB of free device memory")
    tile = synth.to_rgbx(synth.noisy(512, 512, 0.15, 3)[1])
    big = torch.from_numpy(tile).cuda().repeat((H + 511) // 512, W // 512, 1)[:H].contiguous()
    out = vf.filter(big, criterion=crit, window=w, approx=approx, degree=4)
    torch.cuda.synchronize()
    del big
    R = w // 2
    row4g = (2 ** 32) // (W * 4)  # first row past the 4 GiB offset
    cols = np.arange(W) % 512
    for r0, r1 in [(0, 2), (row4g - 1, row4g + 2), (H - 2, H)]:
        lo, hi = max(r0 - R, 0), min(r1 + R, H)
        sub = tile[np.arange(lo, hi) % 512][:, cols]
        o, d = F.filter_image(sub, F.Config(crit, w, approx, 4), threads=8,
                              rows=(r0 - lo, r1 - lo))
        sl = slice(r0 - lo, r1 - lo)
        g = out[r0:r1].cpu().numpy()
        check(crit, o[sl], {k: v[sl] for k, v in d.items()}, g)
    del out
    torch.cuda.empty_cache()
