"""The paper's printed coefficients on the GPU: vf_set_coefficients loads
Table 1 (the arccos pair, Sec. 3.1) and Table 2 (exp(-z), Sec. 3.2) into the
context, and the CUDA filters evaluating them meet the parity bar against the
FP64 oracle evaluating the same printed rows (oracle Config coeffs="paper")."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import filters as F  # noqa: E402
from oracle import paper_tables as PT  # noqa: E402
from paper_1009_0959_gb300 import synth  # noqa: E402

from test_gpu_parity import check, run_gpu  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0959_gb300 import build, vfilt
    build.build()
    return vfilt


@pytest.fixture
def table1(vf):
    vf.set_coefficients("acos_lo", "poly", 4, PT.TABLE1_ARCCOS, lo=0.0, hi=0.5)
    vf.set_coefficients("acos_hi", "poly", 4, PT.TABLE1_ARCSIN, lo=0.0, hi=2 ** -0.5)
    yield
    vf.set_coefficients("acos_lo", "poly", 4)
    vf.set_coefficients("acos_hi", "poly", 4)


@pytest.fixture
def table2(vf):
    for d, (_, c) in PT.TABLE2_EXP.items():
        vf.set_coefficients("exp", "poly", d, c, lo=0.0, hi=PT.EXP_CUTOFF)
    yield
    for d in PT.TABLE2_EXP:
        vf.set_coefficients("exp", "poly", d)


@pytest.mark.parametrize("w", [3, 5, 7])
@pytest.mark.parametrize("reuse", [1, 0])
def test_bvdf_table1_printed(vf, table1, w, reuse):
    """BVDF with the printed degree-4 Table 1 pair, both kernel paths (the
    pair-reuse tiles and the per-window kernel)."""
    clean, noisy = synth.noisy(45, 77, 0.15, 400 + w)
    o, d = F.filter_image(noisy, F.Config("bvdf", w, "poly", 4, coeffs="paper"))
    try:
        vf.set_option("pair_reuse", reuse)
        g = run_gpu(vf, noisy, criterion="bvdf", window=w, approx="poly", degree=4)
    finally:
        vf.set_option("pair_reuse", 1)
    check("bvdf", o, d, g)


@pytest.mark.parametrize("crit", ["amnfe", "amnfg"])
@pytest.mark.parametrize("deg", [2, 3, 4])
@pytest.mark.parametrize("w", [3, 5])
def test_amnf_table2_printed(vf, table2, crit, deg, w):
    clean, noisy = synth.noisy(45, 77, 0.2, 500 + deg)
    o, d = F.filter_image(noisy, F.Config(crit, w, "poly", deg, coeffs="paper"))
    g = run_gpu(vf, noisy, criterion=crit, window=w, approx="poly", degree=deg)
    check(crit, o, d, g)


def test_caller_rational_through_batch(vf):
    """A caller's (4,4) rational (here the printed tab_exp_rat, loaded as
    VF_MINIMAX_RATIONAL_FIT) in a batched launch: the batch takes the
    coefficients in the context when it is created."""
    vf.set_coefficients("exp", "rational_fit", 4, PT.EXP_RATIONAL_NUM, PT.EXP_RATIONAL_DEN,
                        0.0, PT.EXP_CUTOFF)
    try:
        imgs = []
        for k, w in enumerate((3, 5)):
            clean, noisy = synth.noisy(40 + 7 * k, 90, 0.2, 600 + k)
            t = torch.from_numpy(synth.to_rgbx(noisy)).cuda()
            imgs.append((noisy, t, torch.empty_like(t),
                         dict(criterion="amnfe", window=w, approx="rational_fit", degree=4)))
        b = vf.Batch([(t, o, p) for _, t, o, p in imgs])
        b.launch()
        torch.cuda.synchronize()
        b.close()
    finally:
        vf.set_coefficients("exp", "rational_fit", 4)
    for noisy, _, o, p in imgs:
        ref, d = F.filter_image(noisy, F.Config("amnfe", p["window"], "rational", 4))
        check("amnfe", ref, d, o.cpu().numpy())
