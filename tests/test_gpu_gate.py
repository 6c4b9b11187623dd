"""The learned impulse gate: gradients and forward against the FP64 oracle
(oracle/gate.py), deterministic and resumable training, the gated filter, and
what the trained gate gains over the plain filter."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gate as G  # noqa: E402
from oracle import metrics as M  # noqa: E402
from paper_1009_0959_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0959_gb300 import build, vfilt
    build.build()
    return vfilt


def batch(n, h, w, seed, p_lo=0.05, p_hi=0.3):
    imgs, tgts = [], []
    for k in range(n):
        p = p_lo + (p_hi - p_lo) * k / max(n - 1, 1)
        clean, noisy = synth.noisy(h, w, p, seed * 100 + k)
        imgs.append(synth.to_rgbx(noisy))
        tgts.append(synth.impulse_mask(clean, noisy))
    return np.stack(imgs), np.stack(tgts)


def test_gradient_and_forward_match_oracle(vf):
    """Same BF16-rounded weights on both sides; the GPU accumulates in FP32."""
    imgs, tgts = batch(2, 19, 27, 1)
    theta = G.init(3)
    theta[G.NPARAM - 17:G.NPARAM] += 0.05  # non-zero biases
    theta32 = theta.astype(np.float32)
    gate = vf.Gate()
    gate.set_params(theta32)
    grad, loss, prob = gate.gradient(torch.from_numpy(imgs).cuda(), torch.from_numpy(tgts).cuda())
    torch.cuda.synchronize()
    wq = G.bf16_round(theta32.astype(np.float64))
    caches = [G.forward(imgs[k], wq) for k in range(2)]
    ts = [tgts[k].astype(np.float64) for k in range(2)]
    ref_g = G.backward(caches, ts, wq)
    np.testing.assert_allclose(loss.item(), G.loss(caches, ts), rtol=1e-5)
    np.testing.assert_allclose(prob.cpu().numpy(), np.stack([c["p"] for c in caches]), atol=2e-6)
    g = grad.cpu().numpy()
    np.testing.assert_allclose(g, ref_g, rtol=2e-3, atol=2e-5 * np.abs(ref_g).max())
    # fused FP32 inference (CUDA cores) = the FP32 forward
    try:
        vf.set_option("gate_tensor_cores", 0)
        for k in range(2):
            t = torch.from_numpy(imgs[k]).cuda()
            _, pr = gate.infer(t, 0.5, prob=torch.empty((19, 27), device="cuda"))
            torch.cuda.synchronize()
            np.testing.assert_allclose(pr.cpu().numpy(), caches[k]["p"], atol=2e-6)
            fl = gate.infer(t, 0.5)
            torch.cuda.synchronize()
            sure = np.abs(caches[k]["p"] - 0.5) > 1e-4
            np.testing.assert_array_equal(fl.cpu().numpy()[sure], (caches[k]["p"] > 0.5)[sure])
    finally:
        vf.set_option("gate_tensor_cores", 1)
    gate.close()


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("shape", [(37, 70), (40, 300), (13, 125), (1, 1), (7, 1), (1, 260)])
def test_tensor_core_inference_matches_bf16_oracle(vf, engine, shape):
    """Both tensor-core engines (1: tcgen05 MMAs into TMEM over rows of 128
    cells, 124 x 6 outputs per tile; 2: warp-level mma, 32 x 16 tiles) round
    activations to BF16 between layers; against the oracle taking the same
    reading the remaining differences are FP32 accumulation order and the
    occasional BF16 rounding flip of an activation: probabilities within
    2e-3, flags equal away from the threshold.  The shapes span several tiles
    of either engine with ragged edges, and images smaller than one tile."""
    H, W = shape
    imgs, tgts = batch(2, H, W, 4)
    theta = G.init(5)
    theta[G.NPARAM - 17:] += 0.03
    gate = vf.Gate()
    gate.set_params(theta.astype(np.float32))
    wq = G.bf16_round(theta.astype(np.float32).astype(np.float64))
    try:
        vf.set_option("gate_tensor_cores", engine)
        for k in range(2):
            ref = G.forward(imgs[k], wq, act_bf16=True)["p"]
            t = torch.from_numpy(imgs[k]).cuda()
            fl, pr = gate.infer(t, 0.5,
                                flags=torch.empty((H, W), dtype=torch.uint8, device="cuda"),
                                prob=torch.empty((H, W), device="cuda"))
            torch.cuda.synchronize()
            np.testing.assert_allclose(pr.cpu().numpy(), ref, atol=2e-3)
            sure = np.abs(ref - 0.5) > 5e-3
            np.testing.assert_array_equal(fl.cpu().numpy()[sure], (ref > 0.5)[sure])
        gate.check()  # no device-side wait gave up
    finally:
        vf.set_option("gate_tensor_cores", 1)
    gate.close()


def _train(vf, gate, imgs, tgts, steps, lr=3e-3, bs=8):
    ti, tt = torch.from_numpy(imgs).cuda(), torch.from_numpy(tgts).cuda()
    loss = torch.zeros(1, device="cuda")
    losses = []
    for s in range(steps):
        k = (s * bs) % len(imgs)
        gate.train_step(ti[k:k + bs], tt[k:k + bs], lr, loss)
        losses.append(loss.item())
    return losses


def test_training_deterministic_and_resumable(vf, tmp_path):
    imgs, tgts = batch(16, 48, 48, 2)
    a, b, c = vf.Gate(7), vf.Gate(7), vf.Gate(7)
    la = _train(vf, a, imgs, tgts, 12)
    lb = _train(vf, b, imgs, tgts, 12)
    assert la == lb
    np.testing.assert_array_equal(a.get_params(), b.get_params())
    assert la[10] < la[0]  # the same batch (k = 0) before and after 10 steps
    _train(vf, c, imgs, tgts, 6)
    c.save(tmp_path / "gate.bin")
    d = vf.Gate(99)
    d.load(tmp_path / "gate.bin")
    assert d.step == 6
    # continue exactly where the 12-step run continued: steps 6..11 use the
    # same batches as in a
    ti, tt = torch.from_numpy(imgs).cuda(), torch.from_numpy(tgts).cuda()
    loss = torch.zeros(1, device="cuda")
    tail = []
    for s in range(6, 12):
        k = (s * 8) % 16
        d.train_step(ti[k:k + 8], tt[k:k + 8], 3e-3, loss)
        tail.append(loss.item())
    assert tail == la[6:]
    np.testing.assert_array_equal(d.get_params(), a.get_params())
    # a corrupted checkpoint is rejected
    raw = bytearray((tmp_path / "gate.bin").read_bytes())
    raw[100] ^= 1
    (tmp_path / "bad.bin").write_bytes(bytes(raw))
    with pytest.raises(vf.VFError):
        d.load(tmp_path / "bad.bin")
    for gte in (a, b, c, d):
        gte.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_gated_filter_identities(vf, mode):
    """Under one VF_OPT_PAIR_REUSE setting (0: per-window kernels, 1: the
    pair-reuse tiles for BVDF) the gated call runs the same body and sums as
    the plain call: all flags set gives the plain filter's bytes, none the
    input, a mix each of them where it belongs; the third counter counts the
    flagged pixels."""
    clean, noisy = synth.noisy(45, 77, 0.2, 5)
    t = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
    kw = dict(criterion="bvdf", window=5, approx="poly", degree=4)
    vf.set_option("pair_reuse", mode)
    vf.set_option("gated_sparse", 0)  # the tile forms
    try:
        plain = vf.filter(t, **kw)
        ones = torch.ones((45, 77), dtype=torch.uint8, device="cuda")
        zeros = torch.zeros_like(ones)
        assert torch.equal(vf.filter_gated(t, ones, **kw), plain)
        assert torch.equal(vf.filter_gated(t, zeros, **kw), t)
        half = torch.from_numpy((np.arange(45 * 77).reshape(45, 77) % 3 == 0).astype(np.uint8))
        half = half.cuda()
        st = torch.zeros(3, dtype=torch.int64, device="cuda")
        mixed = vf.filter_gated(t, half, stats=st, **kw)
        torch.cuda.synchronize()
    finally:
        vf.set_option("pair_reuse", 1)
        vf.set_option("gated_sparse", 200)
    m = half.bool().unsqueeze(-1).expand_as(t)
    assert torch.equal(mixed[m], plain[m]) and torch.equal(mixed[~m], t[~m])
    assert st[2].item() == int(half.sum().item()) and st[0].item() == 45 * 77
    for crit in ("vmf", "amnfe"):
        assert torch.equal(vf.filter_gated(t, ones, criterion=crit, window=3),
                           vf.filter(t, criterion=crit, window=3))


@pytest.mark.parametrize("w", [3, 5, 7])
@pytest.mark.parametrize("approx", ["exact", "poly"])
def test_gated_reuse_sparse_flags(vf, w, approx):
    """BVDF gated in the pair-reuse tiles with flags in one corner block and
    a few scattered pixels (most tiles have none and are copied whole): the
    flagged pixels carry the plain filter's bytes, the rest the input; with no
    flag at all every tile is copied; the counters count every pixel once."""
    h, wd = 130, 150
    clean, noisy = synth.noisy(h, wd, 0.2, 40 + w)
    t = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
    kw = dict(criterion="bvdf", window=w, approx=approx, degree=4)
    plain = vf.filter(t, **kw)
    f = np.zeros((h, wd), np.uint8)
    f[:9, :13] = 1
    f[100, 140] = f[64, 3] = f[129, 149] = 1
    flags = torch.from_numpy(f).cuda()
    st = torch.zeros(3, dtype=torch.int64, device="cuda")
    vf.set_option("gated_sparse", 0)  # the tile form, whatever the flagged fraction
    try:
        out = vf.filter_gated(t, flags, stats=st, **kw)
        none = vf.filter_gated(t, torch.zeros_like(flags), **kw)
        torch.cuda.synchronize()
    finally:
        vf.set_option("gated_sparse", 200)
    m = flags.bool().unsqueeze(-1).expand_as(t)
    assert torch.equal(out[m], plain[m]) and torch.equal(out[~m], t[~m])
    assert torch.equal(none, t)
    assert st.tolist()[0] == h * wd and st.tolist()[2] == int(f.sum())


@pytest.mark.parametrize("crit,w,approx", [("bvdf", 5, "poly"), ("bvdf", 3, "exact"),
                                            ("bvdf", 7, "poly"), ("vmf", 5, "exact"),
                                            ("vmf", 7, "exact"), ("amnfe", 5, "rational"),
                                            ("amnfg", 7, "poly"), ("amnfg", 3, "exact")])
def test_gated_sparse_form(vf, crit, w, approx):
    """VF_OPT_GATED_SPARSE: the compacted list of flagged pixels, one window
    each, gives the per-window gated form's bytes (the same window code on
    the same staged samples) and counters, at any flag density, with no flag
    and with every flag; under a limit the device picks the sparse form for
    a sparse map and the tile form (pair-reuse tiles for BVDF) otherwise."""
    h, wd = 53, 141
    clean, noisy = synth.noisy(h, wd, 0.2, 60 + w)
    t = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
    kw = dict(criterion=crit, window=w, approx=approx, degree=4)
    rng = np.random.default_rng(w)
    maps = {d: torch.from_numpy((rng.random((h, wd)) < d).astype(np.uint8)).cuda()
            for d in (0.0, 0.05, 0.6, 1.0)}

    def run(flags, sparse, reuse):
        vf.set_option("gated_sparse", sparse)
        vf.set_option("pair_reuse", reuse)
        try:
            st = torch.zeros(3, dtype=torch.int64, device="cuda")
            out = vf.filter_gated(t, flags, stats=st, **kw)
            torch.cuda.synchronize()
        finally:
            vf.set_option("gated_sparse", 200)
            vf.set_option("pair_reuse", 1)
        return out, st.tolist()

    for d, flags in maps.items():
        ref, st_ref = run(flags, 0, 0)
        out, st = run(flags, 1000, 0)
        assert torch.equal(out, ref), d
        assert st == st_ref and st[0] == h * wd and st[2] == int(flags.sum().item())
        if d == 0.0:
            assert torch.equal(out, t)
        # under a 30 % limit: the sparse form below it, the tile form above
        auto, st_a = run(flags, 300, 1)
        tiles, st_t = run(flags, 0, 1)
        want, st_w = (out, st) if d <= 0.3 else (tiles, st_t)
        assert torch.equal(auto, want), d
        assert st_a == st_w


def test_gated_sparse_form_large(vf):
    """The sparse form on a 1500 x 2048 image: the compaction's CTAs take
    several rounds of 1,024 pixels each, and above the limit they stop early
    (the tile form then rewrites every pixel).  Forced sparse and the
    per-window tile form agree byte for byte at 5 % flags; under the default
    limit a 50 % map gives the tile form's bytes and a 5 % map the sparse
    form's."""
    h, wd = 1500, 2048
    clean, noisy = synth.noisy(h, wd, 0.15, 77)
    t = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
    kw = dict(criterion="bvdf", window=5, approx="poly", degree=4)
    rng = np.random.default_rng(3)

    def run(flags, sparse, reuse):
        vf.set_option("gated_sparse", sparse)
        vf.set_option("pair_reuse", reuse)
        try:
            st = torch.zeros(3, dtype=torch.int64, device="cuda")
            out = vf.filter_gated(t, flags, stats=st, **kw)
            torch.cuda.synchronize()
        finally:
            vf.set_option("gated_sparse", 200)
            vf.set_option("pair_reuse", 1)
        return out, st.tolist()

    for d in (0.05, 0.5):
        flags = torch.from_numpy((rng.random((h, wd)) < d).astype(np.uint8)).cuda()
        window, st_w = run(flags, 0, 0)
        sparse, st_s = run(flags, 1000, 0)
        assert torch.equal(sparse, window) and st_s == st_w
        assert st_s[0] == h * wd and st_s[2] == int(flags.sum().item())
        tiles, st_t = run(flags, 0, 1)
        # the persistent pair-reuse tiles, many per CTA: the plain filter's
        # bytes where flagged, the input elsewhere
        plain = vf.filter(t, **kw)
        m = flags.bool().unsqueeze(-1).expand_as(t)
        assert torch.equal(tiles[m], plain[m]) and torch.equal(tiles[~m], t[~m])
        auto, st_a = run(flags, 200, 1)
        want, st_want = (sparse, st_s) if d < 0.2 else (tiles, st_t)
        assert torch.equal(auto, want) and st_a == st_want


def test_trained_gate_beats_plain_filter(vf):
    """Trained on the GPU by the library's own kernels, the gate flags the
    impulses; the gated 5 x 5 minimax BVDF keeps the clean pixels untouched
    and scores a higher PSNR than the plain filter on held-out images."""
    imgs, tgts = batch(32, 96, 96, 3)
    gate = vf.Gate(11)
    losses = _train(vf, gate, imgs, tgts, 600, lr=1e-2)
    assert np.mean(losses[-20:]) < 0.4 * np.mean(losses[:5])
    for p in (0.10, 0.25):
        clean, noisy = synth.noisy(256, 256, p, 777)
        t = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
        flags = gate.infer(t, 0.5)
        kw = dict(criterion="bvdf", window=5, approx="poly", degree=4)
        gated = vf.filter_gated(t, flags, **kw).cpu().numpy()
        plain = vf.filter(t, **kw).cpu().numpy()
        frac = flags.float().mean().item()
        truth = synth.impulse_mask(clean, noisy).mean()
        assert 0.5 * truth < frac < 2.0 * truth + 0.02
        assert M.psnr(clean, gated) > M.psnr(clean, plain)
    gate.close()
