"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Selection filters (VMF, BVDF, EVMF): the selected colour must equal the
oracle's wherever the oracle's best aggregate is more than 1e-5 (relative)
below the best aggregate of a different colour (and, for EVMF, where P_C and
beta_C differ by more than 1e-5 relative).  The FP32 aggregates carry a
relative error of a few 1e-7 (n - 1 terms, each within a few ulp), far inside
that gap.  AMNF: the rounded output must be equal wherever the oracle's
unrounded output is more than 1e-3 from a rounding boundary: the weighted
mean's FP32 error is below 255 x (a few ulp) ~ 1e-4; within the band it may
differ by one level.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import filters as F  # noqa: E402
from paper_1009_0959_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

SEL_GAP = 1e-5
AMNF_GAP = 1e-3


@pytest.fixture(scope="module")
def vf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0959_gb300 import build, vfilt
    build.build()
    return vfilt


def run_gpu(vf, img, channels=4, **kw):
    src = synth.to_rgbx(img) if channels == 4 else np.ascontiguousarray(img[..., :3])
    t = torch.from_numpy(src).cuda()
    out = vf.filter(t, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check(crit, oracle_out, diag, gpu_out):
    o, g = oracle_out[..., :3].astype(int), gpu_out[..., :3].astype(int)
    diff = np.any(o != g, axis=-1)
    if crit in ("amnfe", "amnfg"):
        safe = diag["gap"] > AMNF_GAP
        assert np.abs(o - g).max() <= 1
    else:
        safe = diag["gap"] > SEL_GAP
    bad = diff & safe
    assert bad.sum() == 0, "%d mismatches outside the near-tie band (%d near ties)" % (
        bad.sum(), (~safe).sum())
    return int((~safe).sum())


CASES = [("vmf", "exact", 0), ("bvdf", "exact", 0), ("bvdf", "poly", 2), ("bvdf", "poly", 4),
         ("bvdf", "poly", 6), ("amnfe", "exact", 0), ("amnfe", "poly", 2), ("amnfe", "poly", 4),
         ("amnfe", "poly", 6), ("amnfe", "rational", 4), ("amnfg", "exact", 0),
         ("amnfg", "poly", 4), ("amnfg", "rational", 4), ("evmf", "exact", 0),
         ("evmf", "poly", 3), ("evmf", "poly", 5), ("evmf", "rational", 4),
         # the library's own best (d,d) rationals (GPU) against the oracle's own
         ("amnfe", "rational_fit", 2), ("amnfe", "rational_fit", 4),
         ("amnfg", "rational_fit", 3), ("evmf", "rational_fit", 2), ("evmf", "rational_fit", 4),
         # the generalised entropy vector filter with the angular distance
         ("evbdf", "exact", 0), ("evbdf", "poly", 3), ("evbdf", "poly", 5)]


@pytest.mark.parametrize("w", [3, 5, 7])
@pytest.mark.parametrize("crit,approx,deg", CASES)
def test_parity_small(vf, crit, approx, deg, w):
    """37 x 67 image: several 32 x 4 tiles plus a ragged column and row."""
    clean, noisy = synth.noisy(37, 67, 0.2, 100 + w)
    kw = dict(criterion=crit, window=w, approx=approx, degree=max(deg, 2))
    out_o, d = F.filter_image(noisy, F.Config(crit, w, approx, max(deg, 2)))
    out_g = run_gpu(vf, noisy, **kw)
    check(crit, out_o, d, out_g)
    # the fourth byte is carried through from the centre / selected pixel (0 here)
    assert (out_g[..., 3] == 0).all()


@pytest.mark.parametrize("crit,approx", [("vmf", "exact"), ("bvdf", "poly"), ("amnfe", "rational"),
                                         ("evmf", "exact")])
def test_parity_rgb_odd_pitch(vf, crit, approx):
    """3-byte pixels with a row pitch of 3 W + 1 bytes (unaligned rows)."""
    clean, noisy = synth.noisy(21, 45, 0.25, 7)
    H, W = noisy.shape[:2]
    buf = torch.zeros((H, W * 3 + 1), dtype=torch.uint8, device="cuda")
    inp = buf.as_strided((H, W, 3), (W * 3 + 1, 3, 1))
    inp.copy_(torch.from_numpy(noisy).cuda())
    obuf = torch.zeros_like(buf)
    out = obuf.as_strided((H, W, 3), (W * 3 + 1, 3, 1))
    vf.filter(inp, out, criterion=crit, window=5, approx=approx, degree=4)
    torch.cuda.synchronize()
    out_o, d = F.filter_image(noisy, F.Config(crit, 5, approx, 4))
    check(crit, out_o, d, out.cpu().numpy())
    # the pad byte after each row is untouched
    assert (obuf[:, -1] == 0).all()


@pytest.mark.parametrize("shape", [(1, 1), (1, 40), (40, 1), (2, 3), (5, 70), (3, 33)])
@pytest.mark.parametrize("w", [3, 5, 7])
@pytest.mark.parametrize("crit", ["vmf", "bvdf", "amnfg", "evmf", "evbdf"])
def test_edge_shapes(vf, shape, w, crit):
    """Images smaller than the window and than a tile (replicated borders)."""
    clean, noisy = synth.noisy(shape[0], shape[1], 0.3, 9)
    out_o, d = F.filter_image(noisy, F.Config(crit, w))
    check(crit, out_o, d, run_gpu(vf, noisy, criterion=crit, window=w))


def test_degenerate_colours(vf):
    """Black pixels (zero vectors: cosine 0 by convention), constant and
    two-colour regions, saturated values."""
    img = np.zeros((24, 40, 3), np.uint8)
    img[:, 20:] = 255
    img[::5, ::7] = (255, 0, 0)
    img[10:14, 5:9] = 0
    img[3, 3] = (0, 0, 1)
    for crit, approx in [("vmf", "exact"), ("bvdf", "exact"), ("bvdf", "poly"),
                         ("amnfe", "exact"), ("amnfg", "poly"), ("evmf", "rational")]:
        for w in (3, 5):
            out_o, d = F.filter_image(img, F.Config(crit, w, approx, 4))
            check(crit, out_o, d, run_gpu(vf, img, criterion=crit, window=w, approx=approx))


@pytest.mark.parametrize("crit,approx,deg", [("vmf", "exact", 0), ("bvdf", "exact", 0),
                                             ("bvdf", "poly", 4), ("amnfe", "rational", 4),
                                             ("amnfg", "poly", 5), ("evmf", "exact", 0),
                                             ("evmf", "poly", 4)])
@pytest.mark.parametrize("w", [3, 5])
def test_parity_full_size_sampled(vf, crit, approx, deg, w):
    """1024 x 1024 at 15 % impulses, launched as the benchmark launches it;
    the oracle checks a sample of rows (top and bottom borders, the middle)."""
    clean, noisy = synth.noisy(1024, 1024, 0.15, 3)
    out_g = run_gpu(vf, noisy, criterion=crit, window=w, approx=approx, degree=max(deg, 2))
    cfg = F.Config(crit, w, approx, max(deg, 2))
    for r0, r1 in [(0, 3), (510, 514), (1021, 1024)]:
        out_o, d = F.filter_image(noisy, cfg, rows=(r0, r1))
        sl = slice(r0, r1)
        check(crit, out_o[sl], {k: v[sl] for k, v in d.items()}, out_g[sl])


def test_stats_counters(vf):
    clean, noisy = synth.noisy(64, 96, 0.15, 21)
    st = torch.zeros(3, dtype=torch.int64, device="cuda")
    run = synth.to_rgbx(noisy)
    t = torch.from_numpy(run).cuda()
    vf.filter(t, criterion="evmf", window=3, stats=st)
    torch.cuda.synchronize()
    pixels, ties, switched = st.tolist()
    assert pixels == 64 * 96
    _, d = F.filter_image(noisy, F.Config("evmf", 3))
    ref = int(d["sw"].sum())
    band = int((d["gap"] <= SEL_GAP).sum())
    assert abs(switched - ref) <= band
    assert ties >= 0


@pytest.mark.parametrize("crit,w,approx", [("vmf", 5, "exact"), ("amnfe", 5, "rational"),
                                            ("bvdf", 5, "poly"), ("bvdf", 3, "exact"),
                                            ("evmf", 5, "poly"), ("evmf", 7, "exact"),
                                            ("evbdf", 5, "poly"), ("vmf", 7, "exact")])
def test_stats_counters_every_kernel(vf, crit, w, approx):
    """The device counters from every kernel family (two windows per thread,
    the tall pair-reuse tiles, the EVMF work queue): every pixel counted once,
    and the switched count of the entropy filters within the oracle's near-tie
    band of its own count."""
    clean, noisy = synth.noisy(77, 130, 0.2, 23)
    st = torch.zeros(3, dtype=torch.int64, device="cuda")
    t = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
    out = vf.filter(t, criterion=crit, window=w, approx=approx, degree=4, stats=st)
    torch.cuda.synchronize()
    pixels, ties, switched = st.tolist()
    assert pixels == 77 * 130 and ties >= 0
    o, d = F.filter_image(noisy, F.Config(crit, w, approx, 4))
    check(crit, o, d, out.cpu().numpy())
    if crit.startswith("ev"):
        band = int((d["gap"] <= SEL_GAP).sum())
        assert abs(switched - int(d["sw"].sum())) <= band
    else:
        assert switched == 0


@pytest.mark.parametrize("w", [3, 5, 7])
def test_stats_counters_reuse_evmf(vf, w):
    """The EVMF in the pair-reuse tiles (the switch in the finish phase):
    every pixel counted once, the switched count within the oracle's near-tie
    band, the same counts as the per-window kernels."""
    clean, noisy = synth.noisy(77, 130, 0.2, 29)
    t = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
    counts = []
    try:
        for mode in (2, 0):
            vf.set_option("pair_reuse", mode)
            st = torch.zeros(3, dtype=torch.int64, device="cuda")
            vf.filter(t, criterion="evmf", window=w, approx="poly", degree=4, stats=st)
            torch.cuda.synchronize()
            counts.append(st.tolist())
    finally:
        vf.set_option("pair_reuse", 1)
    _, d = F.filter_image(noisy, F.Config("evmf", w, "poly", 4))
    band = int((d["gap"] <= SEL_GAP).sum())
    for pixels, ties, switched in counts:
        assert pixels == 77 * 130 and ties >= 0
        assert abs(switched - int(d["sw"].sum())) <= band
    assert counts[0][2] == counts[1][2]


def test_minimax_quality_bar(vf):
    """Against the FP64 oracle's exact filter on the 256 x 256, 10 % case:
    the degree-4 arccos (Table 1) changes at most 0.5 % of the selections and
    costs at most 0.05 dB of PSNR; the paper's rationals likewise."""
    from oracle import metrics as M
    clean, noisy = synth.noisy(256, 256, 0.10, 1)
    for crit, approx, deg in [("bvdf", "poly", 4), ("amnfe", "rational", 4),
                              ("evmf", "rational", 4)]:
        ex, _ = F.filter_image(noisy, F.Config(crit, 3), threads=4)
        g = run_gpu(vf, noisy, criterion=crit, window=3, approx=approx, degree=deg)[..., :3]
        assert M.changed_fraction(ex, g) <= 0.005
        assert M.psnr(clean, ex) - M.psnr(clean, g) <= 0.05


def test_evmf_centre_equals_mean(vf):
    """Six samples (98,100,100), two (106,100,100) and the centre
    (100,100,100): the mean equals the centre, P_C = 0 = beta_C, so the
    identity branch is taken, although the vector median would pick
    (98,100,100).  A rounded mean would make P_C > 0 and switch."""
    img = np.zeros((3, 3, 3), np.uint8)
    img[...] = (98, 100, 100)
    img[1, 1] = (100, 100, 100)
    img[0, 2] = img[2, 0] = (106, 100, 100)
    big = np.zeros((5, 5, 3), np.uint8)
    big[...] = (100, 100, 100)
    big[1:4, 1:4] = img
    out_o, d = F.filter_image(big, F.Config("evmf", 3))
    assert d["sw"][2, 2] == 0 and tuple(out_o[2, 2]) == (100, 100, 100)
    vmf, _ = F.filter_image(big, F.Config("vmf", 3))
    assert tuple(vmf[2, 2]) == (98, 100, 100)
    g = run_gpu(vf, big, criterion="evmf", window=3)
    assert tuple(g[2, 2, :3]) == (100, 100, 100)


def test_alias_rejected(vf):
    t = torch.zeros((16, 16, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(vf.VFError) as e:
        vf.filter(t, t)
    assert e.value.name == "VF_ERR_ALIAS"


@pytest.mark.parametrize("w", [3, 5, 7])
@pytest.mark.parametrize("crit,approx,deg", [("vmf", "exact", 4), ("bvdf", "exact", 4),
                                             ("bvdf", "poly", 3), ("amnfe", "poly", 5),
                                             ("amnfg", "rational", 4), ("amnfe", "exact", 4),
                                             ("evbdf", "exact", 4), ("evbdf", "poly", 4),
                                             ("evmf", "exact", 4), ("evmf", "poly", 4),
                                             ("evmf", "rational", 4)])
def test_pair_reuse_and_per_window_agree(vf, crit, approx, deg, w):
    """Both execution paths (pair-reuse tiles and per-window tiles) meet the
    oracle parity bar on the same 75 x 100 image (ragged in both tile
    shapes)."""
    clean, noisy = synth.noisy(75, 100, 0.2, 300 + w)
    o, d = F.filter_image(noisy, F.Config(crit, w, approx, deg))
    try:
        vf.set_option("pair_reuse", 2)
        a = run_gpu(vf, noisy, criterion=crit, window=w, approx=approx, degree=deg)
        vf.set_option("pair_reuse", 0)
        b = run_gpu(vf, noisy, criterion=crit, window=w, approx=approx, degree=deg)
    finally:
        vf.set_option("pair_reuse", 1)
    check(crit, o, d, a)
    check(crit, o, d, b)


def test_graph_capture_matches_eager(vf):
    """vf_filter calls captured in a CUDA graph (every kernel family: per
    window, pair reuse, the EVMF work queue, packed) replay to the same bytes
    as the eager calls."""
    clean, noisy = synth.noisy(70, 150, 0.2, 77)
    src = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
    calls = [dict(criterion="vmf", window=5), dict(criterion="bvdf", window=5),
             dict(criterion="bvdf", window=3, approx="poly", degree=4),
             dict(criterion="amnfe", window=5, approx="rational"),
             dict(criterion="evmf", window=3), dict(criterion="evmf", window=5, approx="poly",
                                                     degree=4),
             dict(criterion="evmf", window=7), dict(criterion="vmf", window=5, precision="fp16x2")]
    eager = [vf.filter(src, **kw) for kw in calls]
    outs = [torch.zeros_like(src) for _ in calls]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            for kw, o in zip(calls, outs):
                vf.filter(src, o, **kw)
    torch.cuda.current_stream().wait_stream(s)
    for o in outs:
        o.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for kw, e, o in zip(calls, eager, outs):
        assert torch.equal(e, o), kw


def test_overlapped_launches_keep_stream_order(vf):
    """A chain of filters, each reading the previous one's output, gives the
    same bytes with programmatic dependent launches (default) as with plain
    launches: every kernel waits for its predecessor before reading."""
    clean, noisy = synth.noisy(300, 260, 0.25, 91)
    src = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
    chain = [dict(criterion="bvdf", window=5, approx="poly", degree=4),
             dict(criterion="evmf", window=5), dict(criterion="vmf", window=3),
             dict(criterion="amnfe", window=5, approx="rational"),
             dict(criterion="bvdf", window=3), dict(criterion="evmf", window=7),
             dict(criterion="vmf", window=5, precision="fp16x2")]

    def run():
        x = src
        for kw in chain:
            x = vf.filter(x, **kw)
        torch.cuda.synchronize()
        return x

    try:
        vf.set_option("overlap_launch", 0)
        plain = run()
    finally:
        vf.set_option("overlap_launch", 1)
    for _ in range(3):
        assert torch.equal(run(), plain)


def test_host_entry_points(vf):
    """vf_filter_host and the pipelined vf_filter_host_async / vf_host_sync
    give the device call's bytes: images of different sizes (the staging
    slots grow), RGB and RGBX, pinned and pageable, more images than slots."""
    cases = [(37, 67, 4, 5, "vmf"), (120, 300, 4, 5, "bvdf"), (64, 64, 3, 3, "amnfe"),
             (200, 150, 4, 7, "evmf"), (33, 97, 3, 5, "amnfg"), (256, 256, 4, 5, "evmf"),
             (17, 40, 4, 3, "bvdf")]
    host_in, expect = [], []
    for k, (h, w, c, win, crit) in enumerate(cases):
        clean, noisy = synth.noisy(h, w, 0.2, 300 + k)
        src = synth.to_rgbx(noisy) if c == 4 else np.ascontiguousarray(noisy)
        t = torch.from_numpy(src)
        host_in.append(t.pin_memory() if k % 2 == 0 else t.clone())
        expect.append(vf.filter(t.cuda(), criterion=crit, window=win, approx="poly",
                                degree=4).cpu())
    torch.cuda.synchronize()
    for (h, w, c, win, crit), t, e in zip(cases, host_in, expect):
        o = vf.filter_host(t, criterion=crit, window=win, approx="poly", degree=4)
        assert torch.equal(o, e)
    outs = [torch.zeros_like(t).pin_memory() for t in host_in]
    for (h, w, c, win, crit), t, o in zip(cases, host_in, outs):
        vf.filter_host_async(t, o, criterion=crit, window=win, approx="poly", degree=4)
    vf.host_sync()
    for o, e in zip(outs, expect):
        assert torch.equal(o, e)
