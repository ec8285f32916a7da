"""The benchmark's multi-GPU path is replicas only: every rank runs its own problem, there is no
data-path collective, and the job's rate is all ranks' units over the slowest rank's time. The
host-side aggregation is checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_seconds = [0.5, 0.8][rank]
    t = bench.max_over_ranks(local_seconds, dist, device="cpu")
    rate = bench.whole_job_rate(10, world, t)
    out[rank] = (t, rate, bench.dist_env())
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()  # no fork of this (threaded) process
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        t, rate, env = out[rank]
        assert t == pytest.approx(0.8)
        assert rate == pytest.approx(2 * 10 / 0.8)
        assert env == (rank, world, 0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload, steps, warmup, restart, gpus = "cube16_cc", 1, 0, 20, 2
    bench.run_reference(A())
    assert capsys.readouterr().out == ""


def test_reference_arm_rank0_prints_the_contract_line(monkeypatch, capsys):
    """The reference arm (the oracle on the host cores) prints one JSON line with the keys the
    benchmark contract names, its e2e equal to its value and no host-device bytes."""
    import json

    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")

    class A:
        workload, steps, warmup, restart, gpus = "cube16_cc", 2, 1, 20, 1
    bench.run_reference(A())
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["config"]["workload"]


def test_oracle_timing_on_a_stretched_grid():
    """The oracle's timing script, as the benchmark calls it beside the stretched line."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-m", "oracle.bench_cpu", "--workload", "cube16_cc", "--evals", "2",
                        "--stretch", "0.12"], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-1000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["value"] > 0 and d["evals"] == 2 and d["stretch"] == 0.12 and d["setup_seconds"] >= 0
