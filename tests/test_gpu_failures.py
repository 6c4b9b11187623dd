"""Allocation failures injected through vf_debug_fail_alloc: each call that
allocates reports VF_ERR_OOM when its allocation is refused, releases what it
had taken, and leaves the context usable; once the countdown lets every
allocation through, the call succeeds with the same results as without the
hook.  Host-side failures only: nothing here faults or stalls the device."""
import pytest
import torch

from paper_1009_0959_gb300 import synth, vfilt

pytestmark = pytest.mark.gpu

OOM = 6


@pytest.fixture(autouse=True)
def _disarm():
    vfilt.debug_fail_alloc(-1)
    yield
    vfilt.debug_fail_alloc(-1)


def _img(h, w, seed):
    return torch.from_numpy(synth.to_rgbx(synth.noisy(h, w, 0.15, seed)[1])).cuda()


def _fails_then_succeeds(make, max_allocs):
    """Arm the hook at k = 0, 1, ... until make() succeeds; every earlier try
    must raise VF_ERR_OOM.  Returns (number of refused tries, result)."""
    for k in range(max_allocs + 1):
        vfilt.debug_fail_alloc(k)
        try:
            out = make()
        except vfilt.VFError as e:
            assert e.status == OOM, e
            assert vfilt.debug_fail_alloc(-1) == -1   # the failure disarmed it
            continue
        vfilt.debug_fail_alloc(-1)
        return k, out
    raise AssertionError("still failing after %d allocations" % max_allocs)


def test_host_staging_oom_then_success():
    """A fresh context (its own thread) has no staging buffer: the refused
    allocation fails vf_filter_host, and the next call allocates it and
    matches the device-buffer filter."""
    import threading
    img = _img(67, 91, 1)
    ref = vfilt.filter(img, criterion="vmf", window=5).cpu()
    host = img.cpu()
    got = {}

    def run():
        vfilt.context()                       # this thread's context first
        vfilt.debug_fail_alloc(0)
        try:
            vfilt.filter_host(host, criterion="vmf", window=5)
        except vfilt.VFError as e:
            got["status"] = e.status
        got["out"] = vfilt.filter_host(host, criterion="vmf", window=5)

    t = threading.Thread(target=run)
    t.start()
    t.join()
    assert got.get("status") == OOM
    assert torch.equal(got["out"], ref)


def test_batch_create_oom_at_every_allocation():
    imgs = [_img(40, 70, 2), _img(33, 129, 3), _img(64, 64, 4)]
    params = [dict(criterion="vmf", window=3), dict(criterion="bvdf", window=5),
              dict(criterion="amnfe", window=7)]
    outs = [torch.empty_like(i) for i in imgs]
    refused, batch = _fails_then_succeeds(
        lambda: vfilt.Batch([(i, o, p) for i, o, p in zip(imgs, outs, params)]), 16)
    assert refused >= 4            # the handle and at least three device buffers
    batch.launch()
    torch.cuda.synchronize()
    for i, o, p in zip(imgs, outs, params):
        assert torch.equal(o, vfilt.filter(i, **p))
    batch.close()


def test_gate_create_and_training_scratch_oom():
    refused, gate = _fails_then_succeeds(lambda: vfilt.Gate(7), 16)
    assert refused >= 7            # the handle and the weight, moment and status buffers
    ref = vfilt.Gate(7)
    assert (gate.get_params() == ref.get_params()).all()
    imgs = torch.stack([_img(24, 40, 5), _img(24, 40, 6)])
    tgt = (torch.rand(imgs.shape[:3], generator=torch.Generator().manual_seed(0)) < 0.3)
    tgt = tgt.to(torch.uint8).cuda()
    # the training scratch is allocated on first use: refuse each of its buffers
    refused, _ = _fails_then_succeeds(lambda: gate.train_step(imgs, tgt, 1e-3), 16)
    assert refused >= 1
    ref.train_step(imgs, tgt, 1e-3)
    torch.cuda.synchronize()
    assert (gate.get_params() == ref.get_params()).all()
    assert gate.step == ref.step == 1
    gate.close()
    ref.close()
