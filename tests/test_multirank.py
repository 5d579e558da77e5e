"""The N > 1 host logic of bench.py on CPU with gloo (world size 2): every
rank runs its own replica, the job's time is the slowest rank's (an
all-reduce MAX), and the whole-job throughput counts every rank's work; the
reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank               # rank 1 is the slower replica
        t_max = bench.max_over_ranks(local_ms, dist, "cpu")
        value = bench.job_throughput(2.0e12, 3, world, t_max)
        results[rank] = (t_max, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, results), nprocs=world, join=True)
        res = dict(results)
    assert set(res) == {0, 1}
    for rank in range(world):
        t_max, value = res[rank]
        assert t_max == 150.0                          # the slowest rank's time on every rank
        # 2 replicas x 3 steps x 2 TFLOP in 0.15 s
        assert value == pytest.approx(2 * 3 * 2.0e12 / 0.15 / 1e9)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.job_throughput(1.0e9, 2, 1, 1000.0) == pytest.approx(2.0)


def test_reference_arm_other_ranks_exit_without_work(capsys):
    import bench

    class Args:
        steps = 1
        warmup = 0
    assert bench.run_reference(Args(), rank=1, world=2) == 0
    assert capsys.readouterr().out == ""
