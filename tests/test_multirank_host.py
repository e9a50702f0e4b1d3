"""The multi-rank path of bench.py on the CPU: two gloo ranks, each with its
own problem size, combine their step times by max over ranks and report the
whole-job weak-scaling throughput (no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [12.5, 40.0][rank]                   # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, "cpu")
        out[rank] = (ms, bench.weak_value(1000, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_value():
    world, port = 2, _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 40.0
        assert value == pytest.approx(2 * 1000 / 0.040)


def test_single_process_is_a_no_op():
    import bench
    assert bench.max_over_ranks(7.0, "cpu") == 7.0
    assert bench.weak_value(500, 1, 250.0) == pytest.approx(2000.0)


def test_strong_value_counts_the_one_problem_once():
    import bench
    # one sharded problem of 3000 units finished by the slowest rank in 250 ms
    assert bench.strong_value(3000, 250.0) == pytest.approx(12000.0)
