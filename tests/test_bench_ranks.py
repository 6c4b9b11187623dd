"""Host logic of the benchmark's multi-GPU form (replicas: every rank filters
its own images, no data-path collective) on CPU with two gloo ranks: the
timing reduction takes the slowest rank, the whole-job throughput counts the
pixels of every rank, each rank's images come from their own seeds, and the
reference arm runs on rank 0 only."""
import contextlib
import io
import os
import socket
import types

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(10.0 + 3.5 * rank, dist, "cpu")
        seeds = [bench.rank_seed(s, rank) for s, _ in [(2, 0), (3, 0), (4, 0)]]
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        q.put((rank, slowest, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    torch.multiprocessing.spawn(_worker, args=(2, _free_port(), q), nprocs=2, join=True)
    results = sorted(q.get(timeout=60) for _ in range(2))
    assert [r for r, _, _ in results] == [0, 1]
    for _, slowest, gathered in results:
        assert slowest == 13.5  # every rank reports the slowest rank's time
        flat = [s for seeds in gathered for s in seeds]
        assert len(set(flat)) == len(flat)  # no image is filtered by two ranks


def test_single_process_helpers():
    assert bench.max_over_ranks(7.25) == 7.25
    assert bench.rank_seed(2, 0) == 2
    # 176 Mpix per rank and step, 5 steps, 2 ranks, 2 s: 880 Mpix/s for the job
    assert bench.job_throughput(176e6, 5, 2, 2000.0) == pytest.approx(880.0)


def test_reference_arm_runs_on_rank_zero_only():
    args = types.SimpleNamespace(steps=1, warmup=0)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        assert bench.reference_arm(args, 1, 2) == 0
    assert out.getvalue() == ""


def test_bench_lab_matches_oracle_metrics():
    """The benchmark's quality study converts to L*a*b* with its own code
    (numpy and torch forms); both agree with the oracle's pinned conversion
    (oracle.metrics.srgb_to_lab: sRGB white -> (100, 0, 0)) on every 8-bit
    grey level and on random colours, and so do the NCD figures built on it."""
    import numpy as np
    from oracle import metrics as M
    rng = np.random.default_rng(3)
    rgb = np.concatenate([np.repeat(np.arange(256, dtype=np.uint8)[:, None], 3, 1),
                          rng.integers(0, 256, (4096, 3)).astype(np.uint8)])
    ref = M.srgb_to_lab(rgb)
    np.testing.assert_allclose(bench._lab(rgb), ref, rtol=0, atol=1e-10)
    got = bench._lab_torch(torch.from_numpy(rgb)).numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9)
    clean = rng.integers(0, 256, (40, 50, 3)).astype(np.uint8)
    other = np.clip(clean.astype(int) + rng.integers(-9, 10, clean.shape), 0, 255).astype(np.uint8)
    lc = bench._lab(clean)
    ncd = np.linalg.norm(bench._lab(other) - lc, axis=-1).sum() / np.linalg.norm(lc, axis=-1).sum()
    assert ncd == pytest.approx(M.ncd(clean, other), rel=1e-12)


def test_roofline_object():
    """The roofline's arithmetic: FP32 ops per pixel x pixels / launch time
    against 152 x 128 lanes x the maximum clock; the issue fraction against
    the same rate; traffic = DRAM bytes per pixel x pixels."""
    r = bench.roofline("bvdf/exact/w5", {"fp32": 1000, "inst": 3000, "dram": 7.0,
                                         "fma_pipe": 0.4}, 1 << 20, 0.1, None)
    peak = r["peak"]
    assert peak == pytest.approx(152 * 128 * 2070e6 / 1e12, rel=1e-3)
    assert r["achieved"] == pytest.approx(1000 * (1 << 20) / 1e-4 / 1e12, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / peak, rel=1e-3)
    assert r["issue_frac"] == pytest.approx(3 * r["frac"], rel=1e-3)
    assert r["traffic"] == 7 * (1 << 20) and r["bound"] == "alu"
    empty = bench.roofline("x", None, 100, 1.0, 2000.0)
    assert empty["frac"] is None and empty["traffic"] is None


def test_clock_summary():
    """The clock record of the result line from nvidia-smi's csv,noheader,
    nounits lines: median SM clock, the largest maximum clock, every throttle
    reason seen Active (sw_power_cap here), peak power ([N/A] skipped)."""
    lines = [
        "0, 2070, 2070, 220.76, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1965, 2070, 1390.12, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2070, 2070, [N/A], 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "garbage line\n",
    ]
    ck = bench.clock_summary(lines)
    assert ck["sm_mhz"] == 2070.0 and ck["sm_max_mhz"] == 2070.0
    assert ck["reasons"] == ["sw_power_cap"] and ck["samples"] == 3
    assert ck["power_w_max"] == 1390.12
    hot = bench.clock_summary([lines[0].replace("Not Active, Not Active, Not Active, Not Active",
                                                "Active, Not Active, Active, Not Active")])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.clock_summary([])["reasons"] == ["no samples"]


def test_clocks_without_nvidia_smi(monkeypatch):
    """Where nvidia-smi cannot be started the record says so instead of
    failing the run."""
    def no_smi(*a, **k):
        raise OSError("nvidia-smi not found")
    monkeypatch.setattr(bench.subprocess, "Popen", no_smi)
    c = bench.Clocks(0)
    c.start()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_failed_side_section_keeps_the_line():
    """A side section that raises is recorded as {"error": ...} in its place;
    the summary of the others is still built."""
    sections = {"per_filter_window": {
        "vmf/w3": {"exact_mpix_s": 100.0, "best_minimax": None},
        "bvdf/w5": {"exact_mpix_s": 10.0, "best_minimax": "poly3",
                    "poly3": {"mpix_s": 11.0, "speedup": 1.1}}}}
    bench.run_section(sections, "batched", lambda: {"mpix_s": 5.0, "speedup_vs_per_image": 1.05})

    def boom():
        raise RuntimeError("CUDA error: an illustrative failure\nsecond line")
    bench.run_section(sections, "precision", boom)
    bench.run_section(sections, "gate", lambda: {
        "speedup_gated_vs_plain": 0.74, "psnr_gated_db_mean": 33.3, "psnr_plain_db_mean": 33.0,
        "flagged_fraction_mean": 0.36,
        "per_frame_forms": [{"flagged": 0.3, "plain_ms": 1.0, "gate_ms": 0.2, "gated_default_ms": 0.9},
                            {"flagged": 0.1, "plain_ms": 1.0, "gate_ms": 0.2, "gated_default_ms": 0.6}]})
    assert sections["precision"] == {"error": "RuntimeError: CUDA error: an illustrative failure"}
    out = bench.summarize(sections)
    assert out["per_filter_window"]["bvdf/w5"] == [10.0, "poly3", 11.0, 1.1]
    assert out["per_filter_window"]["vmf/w3"] == [100.0, None, None, None]
    assert out["batched"] == {"mpix_s": 5.0, "speedup_vs_per_image": 1.05}
    assert out["precision"] == sections["precision"]
    assert out["gate"]["cleanest_frame"] == {"flagged": 0.1, "speedup_vs_plain": 1.25}
    assert out["gate"]["psnr_gain_db"] == 0.3
