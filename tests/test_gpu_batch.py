"""The batched persistent launch (vf_batch_*): every image of a mixed batch
matches the FP64 oracle with the single-image parity bar; plain launch, CUDA
graph replay and the autotuned configuration give identical bytes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import filters as F  # noqa: E402
from paper_1009_0959_gb300 import synth  # noqa: E402

from test_gpu_parity import check  # noqa: E402

pytestmark = pytest.mark.gpu

CRITS = ["vmf", "bvdf", "amnfe", "amnfg", "evmf"]
MINIMAX = {"vmf": ("exact", 4), "bvdf": ("poly", 4), "amnfe": ("rational", 4),
           "amnfg": ("poly", 3), "evmf": ("poly", 5)}


@pytest.fixture(scope="module")
def vf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0959_gb300 import build, vfilt
    build.build()
    return vfilt


def make_batch(n, seed, lo=(1, 1), hi=(70, 90)):
    sizes = synth.batch_sizes(n, seed, lo=lo, hi=hi)
    items = []
    for i, (h, w) in enumerate(sizes):
        crit = CRITS[i % 5]
        win = (3, 5, 7)[i % 3]
        approx, deg = ("exact", 4) if (i // 5) % 2 == 0 else MINIMAX[crit]
        clean, noisy = synth.noisy(h, w, 0.05 + 0.25 * (i % 4) / 3, seed * 100 + i)
        items.append((noisy, dict(criterion=crit, window=win, approx=approx, degree=deg)))
    return items


def to_dev(items, channels=4):
    dev = []
    for noisy, params in items:
        src = synth.to_rgbx(noisy) if channels == 4 else noisy
        t = torch.from_numpy(np.ascontiguousarray(src)).cuda()
        dev.append((t, torch.zeros_like(t), params))
    return dev


def test_batch_matches_oracle(vf):
    items = make_batch(30, 1)
    dev = to_dev(items)
    b = vf.Batch(dev)
    b.launch()
    torch.cuda.synchronize()
    for (noisy, params), (_, out, _) in zip(items, dev):
        o, d = F.filter_image(noisy, F.Config(params["criterion"], params["window"],
                                              params["approx"], params["degree"]))
        check(params["criterion"], o, d, out.cpu().numpy())
    b.close()


def test_batch_graph_autotune_identical(vf):
    """Within one configuration, plain and graph launches give identical
    bytes; every tile shape the autotuner or the caller picks meets the
    oracle parity bar (with 32 x 8 tiles BVDF runs the pair-reuse body, whose
    sums are in another order, so near ties may resolve differently)."""
    items = make_batch(20, 2, lo=(20, 30), hi=(120, 200))
    dev = to_dev(items)
    refs = [F.filter_image(noisy, F.Config(p["criterion"], p["window"], p["approx"], p["degree"]))
            for noisy, p in items]
    b = vf.Batch(dev)

    def run_and_check():
        b.launch()
        torch.cuda.synchronize()
        first = [o.clone() for _, o, _ in dev]
        for _, o, _ in dev:
            o.zero_()
        b.graph_launch()
        b.graph_launch()
        torch.cuda.synchronize()
        for f, (_, o, p), (ro, rd) in zip(first, dev, refs):
            assert torch.equal(f, o)
            check(p["criterion"], ro, rd, o.cpu().numpy())

    run_and_check()
    cfg = b.autotune()
    assert cfg["tile_rows"] in (2, 4, 8) and cfg["ctas_per_sm"] >= 1 and cfg["ms"] > 0
    assert cfg["pixels_per_thread"] in (0, 1, 2)
    assert cfg["mode"] in ("one_kernel", "class_kernels")
    run_and_check()
    for ty in (2, 8):
        for ppt in (0, 1, 2):
            b.configure(ty, 1, pixels_per_thread=ppt)
            assert b.config() == {"mode": "one_kernel", "tile_rows": ty, "ctas_per_sm": 1,
                                  "pixels_per_thread": ppt}
            run_and_check()
    with pytest.raises(vf.VFError):
        b.configure(4, 0, pixels_per_thread=3)
    b.close()


def test_batch_rgb_and_single_image_agree(vf):
    """3-byte pixels in a batch; every image also equals the single-image call
    outside near ties (the batch runs 5 x 5 through the rolled pair loop)."""
    items = make_batch(10, 3, lo=(8, 8), hi=(60, 80))
    dev = to_dev(items, channels=3)
    b = vf.Batch(dev)
    b.launch()
    torch.cuda.synchronize()
    for (noisy, params), (inp, out, _) in zip(items, dev):
        single = vf.filter(inp, **params)
        torch.cuda.synchronize()
        o, d = F.filter_image(noisy, F.Config(params["criterion"], params["window"],
                                              params["approx"], params["degree"]))
        check(params["criterion"], o, d, out.cpu().numpy())
        check(params["criterion"], o, d, single.cpu().numpy())
    b.close()


def test_batch_errors(vf):
    t = torch.zeros((8, 8, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(vf.VFError) as e:
        vf.Batch([(t, t, {})])
    assert e.value.name == "VF_ERR_ALIAS"
    o = torch.zeros_like(t)
    with pytest.raises(vf.VFError) as e:
        vf.Batch([(t, o, {"window": 9})])
    assert e.value.name == "VF_ERR_UNSUPPORTED"
    b = vf.Batch([(t, o, {})])
    with pytest.raises(vf.VFError):
        b.configure(3, 1)
    b.close()


def test_batch_class_kernels(vf):
    """The class-kernel form (one persistent kernel per class, concurrent
    branches): every image meets the oracle parity bar; plain and graph
    launches give the same bytes; VMF, AMNF and BVDF images (the single-image
    kernels' bodies and tile shapes) equal the single-image call byte for
    byte."""
    items = make_batch(40, 4, lo=(1, 1), hi=(150, 230))
    dev = to_dev(items)
    b = vf.Batch(dev)
    b.set_mode("class_kernels")
    assert b.config()["mode"] == "class_kernels"
    b.launch()
    torch.cuda.synchronize()
    first = [o.clone() for _, o, _ in dev]
    for _, o, _ in dev:
        o.zero_()
    b.graph_launch()
    b.graph_launch()
    torch.cuda.synchronize()
    for (noisy, p), (inp, o, _), f in zip(items, dev, first):
        assert torch.equal(f, o)
        ro, rd = F.filter_image(noisy, F.Config(p["criterion"], p["window"], p["approx"],
                                                p["degree"]))
        check(p["criterion"], ro, rd, o.cpu().numpy())
        if p["criterion"] != "evmf":
            single = vf.filter(inp, **p)
            torch.cuda.synchronize()
            assert torch.equal(single, o), p
    b.set_mode("one_kernel")
    b.launch()
    torch.cuda.synchronize()
    for (noisy, p), (_, o, _) in zip(items, dev):
        ro, rd = F.filter_image(noisy, F.Config(p["criterion"], p["window"], p["approx"],
                                                p["degree"]))
        check(p["criterion"], ro, rd, o.cpu().numpy())
    with pytest.raises(vf.VFError):
        lib_set_mode(vf, b, 7)  # no such form
    b.close()


def lib_set_mode(vf, b, mode):
    st = vf.lib().vf_batch_set_mode(b.handle, mode)
    if st != 0:
        raise vf.VFError(st, "bad mode")
