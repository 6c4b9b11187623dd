"""The allocation-free batched call (vf_batch_run_static).

Some callers may not allocate GPU memory while they filter, e.g. a real-time
video pipeline or a plug-in inside an application that reserves all device
memory up front: cudaMalloc there can stall the device for an unbounded time.
This entry point keeps its scratch in a fixed array inside the library.  The
test calls it through the C ABI twice in a row and checks both results against
the ordinary batched call (vf_batch_create + vf_batch_launch) on the same
images: the same kernel and tiles, so the bytes must be identical (a stricter
bar than the near-tie band of the parity tests).  This file is collected last
so that a run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1009_0959_gb300 import synth  # noqa: E402

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


def _images(n, seed):
    sizes = synth.batch_sizes(n, seed, lo=(1, 1), hi=(90, 150))
    out = []
    for i, (h, w) in enumerate(sizes):
        crit = CRITS[i % 5]
        approx, deg = ("exact", 4) if (i // 5) % 2 == 0 else MINIMAX[crit]
        params = dict(criterion=crit, window=(3, 5, 7)[i % 3], approx=approx, degree=deg)
        noisy = synth.noisy(h, w, 0.2, seed * 1000 + i)[1]
        t = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
        out.append((t, params))
    return out


def test_static_batch_matches_batch_twice(vf):
    imgs = _images(40, 5)
    ref = [(t, torch.zeros_like(t), p) for t, p in imgs]
    b = vf.Batch(ref)  # also fits and caches the polynomial approximants
    b.launch()
    torch.cuda.synchronize()
    for call in range(2):
        outs = [(t, torch.full_like(t, 7), p) for t, p in imgs]
        st = vf.batch_run_static(outs)
        assert st == 0, vf.status_string(st)
        torch.cuda.synchronize()
        for (_, r, _), (_, o, _) in zip(ref, outs):
            assert torch.equal(r, o), "call %d differs from vf_batch_launch" % call
    b.close()


def test_static_batch_limits(vf):
    t = torch.zeros((4, 4, 4), dtype=torch.uint8, device="cuda")
    o = torch.zeros_like(t)
    too_many = [(t, o, {})] * (vf.STATIC_MAX_IMAGES + 1)
    assert vf.status_string(vf.batch_run_static(too_many)) == "unsupported combination"
    assert vf.batch_run_static([(t, t, {})]) == 2  # VF_ERR_ALIAS
    assert vf.batch_run_static([(t, o, {"window": 9})]) == 3


def test_static_batch_rational_fits(vf):
    """The library's own rationals in the allocation-free call: they must be
    in the context's cache (an ordinary call fits them), else the call is
    refused before anything is launched; once fitted, the call gives the
    ordinary batched call's bytes."""
    noisy = synth.noisy(40, 70, 0.2, 77)[1]
    t = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
    params = [dict(criterion="amnfe", window=5, approx="rational_fit", degree=3, exp_cutoff=7.5),
              dict(criterion="evmf", window=3, approx="rational_fit", degree=2)]
    outs = [(t, torch.zeros_like(t), p) for p in params]
    assert vf.batch_run_static(outs[:1]) == 3  # not fitted yet: VF_ERR_UNSUPPORTED
    ref = [(t, torch.zeros_like(t), p) for p in params]
    b = vf.Batch(ref)  # fits and caches both rationals
    b.launch()
    torch.cuda.synchronize()
    assert vf.batch_run_static(outs) == 0
    torch.cuda.synchronize()
    for (_, o, _), (_, r, _) in zip(outs, ref):
        assert torch.equal(o, r)
    b.close()


def test_static_batch_bad_enums_and_cutoffs(vf):
    """The same status codes as the ordinary calls for the same bad input: a
    precision outside the enum is VF_ERR_ARG (1), an FP16x2 image
    VF_ERR_UNSUPPORTED (3), an EVMF with a fitted ENT rational and a cut-off
    outside (0, 1) VF_ERR_ARG."""
    t = torch.zeros((8, 8, 4), dtype=torch.uint8, device="cuda")
    o = torch.zeros_like(t)
    assert vf.batch_run_static([(t, o, {"precision": 7})]) == 1
    assert vf.batch_run_static([(t, o, {"criterion": "vmf", "precision": "fp16x2"})]) == 3
    assert vf.batch_run_static([(t, o, dict(criterion="evmf", approx="rational_fit", degree=2,
                                            ent_cutoff=1.5))]) == 1


def test_static_batch_refuses_capture(vf):
    """A call on a capturing stream is refused (VF_ERR_UNSUPPORTED) and leaves
    the capture usable; the plain call afterwards still works."""
    imgs = _images(6, 9)
    ref = [(t, torch.zeros_like(t), p) for t, p in imgs]
    b = vf.Batch(ref)
    b.launch()
    torch.cuda.synchronize()
    outs = [(t, torch.zeros_like(t), p) for t, p in imgs]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    codes = []
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            codes.append(vf.batch_run_static(outs, stream=s))
    torch.cuda.current_stream().wait_stream(s)
    assert codes == [3]
    assert vf.batch_run_static(outs) == 0
    torch.cuda.synchronize()
    for (_, o, _), (_, r, _) in zip(outs, ref):
        assert torch.equal(o, r)
    b.close()


def test_static_batch_back_to_back_on_one_stream(vf):
    """Two calls on the current stream with different image sets, windows and
    criteria and no host wait between them: the second call's descriptor
    copies must not disturb the first call's (each copy has read the host
    staging before its call returns, and calls on one stream are ordered).
    One synchronize, then both outputs byte for byte against the ordinary
    batched call."""
    a = _images(24, 11)
    b_imgs = [(t, dict(p, window={3: 7, 5: 3, 7: 5}[p["window"]],
                       criterion=CRITS[(CRITS.index(p["criterion"]) + 2) % 5]))
              for t, p in _images(30, 12)]
    for p in [p for _, p in b_imgs]:  # keep the minimax settings valid for the new criterion
        p["approx"], p["degree"] = ("exact", 4) if p["approx"] == "exact" else MINIMAX[p["criterion"]]
    refs = []
    for imgs in (a, b_imgs):
        r = [(t, torch.zeros_like(t), p) for t, p in imgs]
        bb = vf.Batch(r)
        bb.launch()
        torch.cuda.synchronize()
        bb.close()
        refs.append(r)
    outs = [[(t, torch.full_like(t, 3), p) for t, p in imgs] for imgs in (a, b_imgs)]
    assert vf.batch_run_static(outs[0]) == 0
    assert vf.batch_run_static(outs[1]) == 0
    torch.cuda.synchronize()
    for out, ref in zip(outs, refs):
        for (_, o, _), (_, r, _) in zip(out, ref):
            assert torch.equal(o, r)
