"""Row bands (one image split over several GPUs or calls; Sec. 3: every
output pixel depends on its own window only).  CPU tests: the band plan of
the C ABI (vf_band_plan) covers every output row exactly once with the halo
it needs, and two gloo ranks that each filter their own band -- with the FP64
oracle as the per-band filter -- into a shared output reproduce the
whole-image filter byte for byte.  The GPU form (bands through vf_filter on
one device, compared with the whole-image call) is tests/test_gpu_bands.py."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402


@pytest.fixture(scope="module")
def vf():
    from paper_1009_0959_gb300 import build
    build.build()
    from paper_1009_0959_gb300 import vfilt
    return vfilt


@pytest.mark.parametrize("H", [1, 2, 7, 37, 1024, 4099])
@pytest.mark.parametrize("window", [3, 5, 7])
@pytest.mark.parametrize("quantum", [1, 4, 8, 14, 16, 20])
def test_band_plan_covers_rows(vf, H, window, quantum):
    h = window // 2
    for bands in sorted({1, 2, 3, 8, min(H, 5), H if H <= 8 else 8}):
        if bands > H:
            continue
        nxt = 0
        for b in range(bands):
            a, n, r0, m = vf.band_plan(H, window, quantum, bands, b)
            assert r0 == nxt and m >= 1  # consecutive, disjoint, non-empty
            nxt = r0 + m
            assert a == 0 or a % quantum == 0
            assert a <= max(0, r0 - h) and a > r0 - h - quantum  # the halo, rounded down
            assert a + n == min(H, r0 + m + h)  # the halo below, clipped
        assert nxt == H


def test_band_plan_errors(vf):
    for args in [(0, 3, 4, 1, 0), (10, 4, 4, 1, 0), (10, 3, 0, 1, 0), (10, 3, 4, 11, 0),
                 (10, 3, 4, 2, 2), (10, 3, 4, 2, -1), (10, -3, 4, 1, 0)]:
        with pytest.raises(vf.VFError):
            vf.band_plan(*args)


def test_row_quantum(vf):
    """The quantum is the tile height of the kernel vf_filter would run."""
    assert vf.row_quantum(criterion="bvdf", window=5) == 20  # pair-reuse tall tiles
    assert vf.row_quantum(criterion="bvdf", window=3) == 14
    assert vf.row_quantum(criterion="bvdf", window=7) == 16
    assert vf.row_quantum(criterion="vmf", window=5) == 8    # two windows per thread, TY 4
    assert vf.row_quantum(criterion="evmf", window=5) == 8   # the work queue's tiles
    assert vf.row_quantum(criterion="evmf", window=3) == 4
    assert vf.row_quantum(criterion="vmf", window=5, precision="fp16x2") == 4
    with pytest.raises(vf.VFError):
        vf.row_quantum(criterion="vmf", window=9)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASES = [("vmf", 5, "exact"), ("bvdf", 3, "poly"), ("amnfe", 7, "rational"), ("evmf", 5, "exact")]


def _band_worker(rank, world, port, path, shape):
    """Rank `rank` filters band `rank` of the image in `path` + '.in' into the
    shared output `path` + '.<case>' (no data moves between the ranks; the
    barrier only orders the check after every band is written)."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import filters as F
        from paper_1009_0959_gb300 import vfilt
        img = np.memmap(path + ".in", np.uint8, "r", shape=shape)
        for k, (crit, w, approx) in enumerate(CASES):
            out = np.memmap(path + ".%d" % k, np.uint8, "r+", shape=shape)
            q = vfilt.row_quantum(criterion=crit, window=w, approx=approx)
            a, n, r0, m = vfilt.band_plan(shape[0], w, q, world, rank)
            local = np.array(img[a:a + n])  # the band's rows, copied locally first
            y, _ = F.filter_image(local, F.Config(crit, w, approx, 4))
            out[r0:r0 + m] = y[r0 - a:r0 - a + m]
            out.flush()
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_bands_reproduce_whole_image():
    from oracle import filters as F
    from paper_1009_0959_gb300 import synth
    _, noisy = synth.noisy(53, 41, 0.2, 61)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "img")
        np.memmap(path + ".in", np.uint8, "w+", shape=noisy.shape)[:] = noisy
        for k in range(len(CASES)):
            np.memmap(path + ".%d" % k, np.uint8, "w+", shape=noisy.shape)[:] = 0
        torch.multiprocessing.spawn(_band_worker, args=(2, _free_port(), path, noisy.shape),
                                    nprocs=2, join=True)
        for k, (crit, w, approx) in enumerate(CASES):
            whole, _ = F.filter_image(noisy, F.Config(crit, w, approx, 4))
            got = np.array(np.memmap(path + ".%d" % k, np.uint8, "r", shape=noisy.shape))
            np.testing.assert_array_equal(got, whole)
