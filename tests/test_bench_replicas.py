"""The N > 1 path of bench.py on the CPU: replicas are timed by the slowest
rank (all_reduce MAX over a gloo group of two processes) and the job's rate
counts every rank's steps; the reference arm runs on rank 0 only."""
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, outdir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    seconds = [3.0, 5.0][rank]  # rank 1 is the slow replica
    slowest = bench.max_over_ranks(seconds, 2)
    rate = bench.replica_rate(4, slowest, 2)
    with open(os.path.join(outdir, f"r{rank}"), "w") as f:
        f.write(f"{slowest} {rate}")
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    tmp.spawn(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in (0, 1):
        slowest, rate = map(float, open(tmp_path / f"r{r}").read().split())
        assert slowest == 5.0
        assert rate == pytest.approx(2 * 4 / 5.0)


def test_single_rank_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.replica_rate(3, 1.5, 1) == 2.0


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench
    args = types.SimpleNamespace(steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args, 1) is None


def test_reference_line_reports_the_sample_and_the_extrapolated_rate(monkeypatch):
    """ms_per_step is the wall time of one bench step (the measured oracle
    sample), value the full-workload rate extrapolated from it by bonds."""
    sys.path.insert(0, ROOT)
    import bench
    calls = []

    def fake_sample(d_sample: int = 4):
        calls.append(d_sample)
        return 2.0, 2.0 * (32 - 1) / (d_sample - 1)

    monkeypatch.setattr(bench, "oracle_sample_seconds", fake_sample)
    args = types.SimpleNamespace(steps=2, warmup=3, gpus=1)
    line = bench.run_reference(args, 0)
    assert len(calls) == 5  # three untimed warm-up samples, two timed
    assert line["impl"] == "reference"
    assert line["ms_per_step"] == pytest.approx(2000.0)
    assert line["extrapolated_ms_per_step"] == pytest.approx(2000.0 * 31 / 3)
    assert line["value"] == pytest.approx(1.0 / (2.0 * 31 / 3))
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "d=4" in line["cpu_baseline"]["sample"] and line["cpu_baseline"]["kind"] == "oracle"
