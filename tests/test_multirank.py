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
    mgr = mp.Manager()
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
