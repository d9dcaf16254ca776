"""Host logic of bench.py on CPU: two gloo ranks aggregate their timed regions into
whole-job throughput (summed units / max time); the cuFFT comparison product; the
nvidia-smi clock and throttle-reason sampling."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = [2.0, 4.0][rank]
    units = [5, 5][rank]
    value, t, u = bench.aggregate(elapsed, units, dist, "cpu")
    q.put((rank, value, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t, u in out:
        assert t == 4.0 and u == 10.0
        assert value == pytest.approx(10.0 / 4.0)


def test_single_rank_aggregation():
    import bench
    assert bench.aggregate(2.0, 4) == (2.0, 2.0, 4)


def test_cufft_comparison_product_matches_explicit_X():
    """The library-FFT comparison product bench.py times beside the kernels computes X x
    (checked on CPU tensors against the explicit trajectory matrix, for several M >= N)."""
    import numpy as np
    import torch

    import bench
    from oracle import trajectory
    rng = np.random.default_rng(3)
    for N, L in [(17, 5), (100, 63), (1000, 500), (1025, 1000)]:
        f = rng.standard_normal(N)
        K = N - L + 1
        X = trajectory.trajectory_matrix(f, L)
        x = rng.standard_normal(K)
        M0 = 1 << (N - 1).bit_length()
        for M in (M0, 2 * M0):
            for dt, tol in ((torch.float64, 1e-13), (torch.float32, 2e-6)):
                prod = bench.fft_product(f, L, M, dt)
                y = prod(torch.from_numpy(x).to(dt)).double().numpy()
                scale = np.linalg.norm(f) * np.linalg.norm(x)
                assert y.shape == (L,)
                assert np.max(np.abs(y - X @ x)) <= tol * scale, (N, L, M, dt)


def _fake_smi(tmp_path, rows):
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n" + "".join(f"echo '{r}'\n" for r in rows))
    fake.chmod(0o755)
    return str(tmp_path)


def test_clock_sampler_reads_clocks_and_reasons(tmp_path, monkeypatch):
    """The throttle reasons that decide whether a bench run counts, parsed from nvidia-smi's CSV."""
    import bench
    rows = ["0, 2070, 2070, 900.50, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 1965, 2070, 1390.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 800.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"]
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, rows) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    out = s.stop()
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    rows = ["0, 1200, 2070, 1000.00, 0x0000000000000008, Active, Not Active, Active, Not Active"]
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, rows) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    out = s.stop()
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and out["sm_mhz"] == 1200.0


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    out = s.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]
