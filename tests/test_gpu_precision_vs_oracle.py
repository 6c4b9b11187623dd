"""The packed-precision forms (FP16x2 / BF16x2 pair terms, FP32 aggregation)
against the FP64 oracle on the precision workload: one 4096 x 4096 image
with 20 % impulses (seed 8), windows 5 and 7, sampled rows (four bands of
six rows: top border, two interior, bottom border).

For every criterion, window and precision the test measures, against the
oracle's EXACT filter, the fraction of changed output pixels and the PSNR
drop on the sampled rows (printed as a table, and written as JSON where the
environment names a file in VF_PRECISION_REPORT), and it checks that every
selection that differs from the oracle evaluating the SAME approximation is
explained by the format: the oracle's relative gap between the best and the
best different colour is within the format's band (4e-3 FP16, 4e-2 BF16:
a few units of its roundoff 2^-11 / 2^-8).  The fraction of pixels inside
that band is reported beside the changed fraction: it is what keeps a
packed selection filter from the 0.5 % changed-selection bar on images
whose smooth regions hold many near-equal aggregates."""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import filters as F  # noqa: E402
from paper_1009_0959_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

BAND = {"fp32": 1e-5, "fp16x2": 4e-3, "bf16x2": 4e-2}
VARIANTS = [("vmf", "exact"), ("bvdf", "poly"), ("amnfe", "rational"), ("evmf", "rational")]
N = 4096


@pytest.fixture(scope="module")
def vf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0959_gb300 import build, vfilt
    build.build()
    return vfilt


@pytest.fixture(scope="module")
def image():
    clean, noisy = synth.noisy(N, N, 0.20, 8)
    rows = np.concatenate([np.arange(0, 6), np.arange(1360, 1366), np.arange(2730, 2736),
                           np.arange(N - 6, N)])
    return clean, noisy, rows


def _oracle_rows(noisy, cfg, rows):
    """The oracle on the sampled rows: each band of six rows is filtered as a
    crop holding the band and the window's halo rows (the crop's own border
    rows coincide with the image's at the top and bottom bands), with all
    host threads."""
    out = np.zeros((len(rows), N, 3), np.uint8)
    gap = np.zeros((len(rows), N))
    k = 0
    h = cfg.window // 2
    for r0 in (0, 1360, 2730, N - 6):
        a, b = max(0, r0 - h), min(N, r0 + 6 + h)
        o, d = F.filter_image(noisy[a:b], cfg, threads=os.cpu_count() or 1)
        sl = slice(r0 - a, r0 - a + 6)
        out[k:k + 6] = o[sl, :, :3]
        g = d["gap"][sl]
        if cfg.criterion in ("amnfe", "amnfg"):
            y = d["yreal"][sl]
            g = np.abs(y - np.floor(y) - 0.5).min(-1)  # distance to a rounding boundary
        gap[k:k + 6] = g
        k += 6
    return out, gap


def _psnr(clean, x):
    mse = ((clean.astype(np.float64) - x.astype(np.float64)) ** 2).mean()
    return 10 * math.log10(255 ** 2 / mse) if mse > 0 else float("inf")


def test_precision_forms_against_oracle(vf, image):
    clean, noisy, rows = image
    t = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
    report = {}
    for w in (5, 7):
        for crit, approx in VARIANTS:
            exact, _ = _oracle_rows(noisy, F.Config(crit, w), rows)
            same, gap = _oracle_rows(noisy, F.Config(crit, w, approx, 4), rows)
            ps_exact = _psnr(clean[rows], exact)
            for prec in ("fp32", "fp16x2", "bf16x2"):
                g = vf.filter(t, criterion=crit, window=w, approx=approx, degree=4,
                              precision=prec)
                torch.cuda.synchronize()
                g = g.cpu().numpy()[rows][..., :3]
                changed = float(np.any(g != exact, axis=-1).mean())
                band = BAND[prec]
                if crit in ("amnfe", "amnfg"):
                    # FP32 and FP16 (exact integer L1 terms): one level, only
                    # within 1e-3 of a rounding boundary; BF16 (L1 terms
                    # rounded to 8 bits): within 8 levels
                    diff = np.abs(g.astype(int) - same.astype(int)).max(-1)
                    if prec == "bf16x2":
                        unexplained = int((diff > 8).sum())
                    else:
                        unexplained = int(((diff > 1) | ((diff == 1) & (gap > 1e-3))).sum())
                    band = 1e-3
                else:
                    unexplained = int((np.any(g != same, axis=-1) & (gap > band)).sum())
                key = "%s/%s/w%d/%s" % (crit, approx, w, prec)
                report[key] = {"changed_vs_oracle_exact": round(changed, 5),
                               "psnr_drop_db": round(ps_exact - _psnr(clean[rows], g), 4),
                               "in_format_band": round(float((gap <= band).mean()), 5),
                               "unexplained": unexplained}
                assert unexplained == 0, (key, unexplained)
    path = os.environ.get("VF_PRECISION_REPORT")
    if path:
        with open(path, "w") as fh:
            json.dump(report, fh, indent=1)
    print("\nvariant changed_vs_oracle_exact psnr_drop_db in_format_band")
    for k, v in report.items():
        print(k, v["changed_vs_oracle_exact"], v["psnr_drop_db"], v["in_format_band"])
    # the FP32 forms of VMF, AMNFE (the paper's rational) and EVMF (the
    # paper's rational) meet the quality bar against the exact filter; the
    # degree-4 arccos changes ~1 % of the BVDF selections here (its own error,
    # not the precision's: the FP32 form is compared), which is reported
    for w in (5, 7):
        for crit, approx in VARIANTS:
            if crit == "bvdf":
                continue
            r = report["%s/%s/w%d/fp32" % (crit, approx, w)]
            assert r["psnr_drop_db"] <= 0.05 and r["changed_vs_oracle_exact"] <= 0.005, (crit, w, r)
