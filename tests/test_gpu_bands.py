"""Row bands on the GPU: an image filtered band by band (each band's rows and
halo copied into device memory of its own, one vf_filter call per band, as
one GPU per band would do it) gives the whole-image call's bytes, for every
kernel family (pair-reuse tiles, two windows per thread, the EVMF work queue,
per-window compaction, packed FP16x2), including the 1024 x 1024 images of
the benchmark."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1009_0959_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0959_gb300 import build, vfilt
    build.build()
    return vfilt


CASES = [dict(criterion="bvdf", window=5), dict(criterion="bvdf", window=3, approx="poly", degree=4),
         dict(criterion="bvdf", window=7, approx="poly", degree=4),
         dict(criterion="vmf", window=5), dict(criterion="vmf", window=7),
         dict(criterion="amnfe", window=5, approx="rational"),
         dict(criterion="amnfg", window=3, approx="poly", degree=4),
         dict(criterion="evmf", window=5), dict(criterion="evmf", window=3, approx="rational"),
         dict(criterion="evmf", window=7, approx="poly", degree=4),
         dict(criterion="evbdf", window=5, approx="poly", degree=4),
         dict(criterion="vmf", window=5, precision="fp16x2"),
         dict(criterion="bvdf", window=5, approx="poly", degree=4, precision="bf16x2")]


@pytest.mark.parametrize("kw", CASES, ids=lambda k: "-".join(str(v) for v in k.values()))
@pytest.mark.parametrize("bands", [2, 3, 7])
def test_bands_match_whole_image(vf, kw, bands):
    _, noisy = synth.noisy(301, 203, 0.2, 71)
    host = torch.from_numpy(synth.to_rgbx(noisy)).pin_memory()
    whole = vf.filter(host.cuda(), **kw).cpu()
    out = torch.zeros_like(host)
    covered = 0
    for b in range(bands):
        out, r0, m = vf.filter_band(host, b, bands, out=out, **kw)
        covered += m
    assert covered == host.shape[0]
    assert torch.equal(out, whole)


@pytest.mark.parametrize("kw", [dict(criterion="bvdf", window=5),
                                dict(criterion="evmf", window=5, approx="poly", degree=4),
                                dict(criterion="vmf", window=3)],
                         ids=["bvdf5", "evmf5", "vmf3"])
def test_bands_full_size(vf, kw):
    """A 1024 x 1024 benchmark image in 8 bands (one per GPU of an 8-GPU node)."""
    _, noisy = synth.noisy(1024, 1024, 0.15, 3)
    host = torch.from_numpy(synth.to_rgbx(noisy)).pin_memory()
    whole = vf.filter(host.cuda(), **kw).cpu()
    out = torch.zeros_like(host)
    for b in range(8):
        out, _, _ = vf.filter_band(host, b, 8, out=out, **kw)
    assert torch.equal(out, whole)
