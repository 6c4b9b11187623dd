"""The per-window kernels' tile height (VF_OPT_TILE_ROWS) is an execution
choice only: each output is its own window's selection or weighted mean
(Sec. 3, problem statement), so 2, 4 and 8 thread rows per CTA give the same
bytes, also across ragged right and bottom tile edges."""
import pytest

torch = pytest.importorskip("torch")

from paper_1009_0959_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [("vmf", "exact", 4), ("amnfe", "exact", 4), ("amnfe", "rational", 4),
         ("amnfg", "poly", 4), ("evmf", "exact", 4), ("evmf", "poly", 3), ("bvdf", "poly", 4)]


@pytest.fixture(scope="module")
def vf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0959_gb300 import build, vfilt
    build.build()
    return vfilt


@pytest.mark.parametrize("window", [3, 5, 7])
def test_tile_rows_do_not_change_outputs(vf, window):
    img = torch.from_numpy(synth.to_rgbx(synth.noisy(777, 1001, 0.15, 5)[1])).cuda().contiguous()
    try:
        for (c, a, d) in CASES:
            outs = {}
            for ty in (4, 2, 8):
                vf.set_option("tile_rows", ty)
                outs[ty] = vf.filter(img, criterion=c, window=window, approx=a, degree=d).cpu()
            for ty in (2, 8):
                assert torch.equal(outs[ty], outs[4]), (c, a, d, window, ty)
    finally:
        vf.set_option("tile_rows", 4)
