"""The N > 1 path of bench.py on the CPU: two gloo ranks agree on the slowest rank's time and the
whole-job throughput counts every rank's updates (weak scaling, one walker per rank)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = 100.0 + 25.0 * rank  # rank 1 is the slow one
        out[rank] = (bench.max_over_ranks(dist, ms, "cpu"),
                     bench.job_throughput(world, 1000, 2, bench.max_over_ranks(dist, ms, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_sum_the_work():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork of a process that already runs threads
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 125.0
        assert value == pytest.approx(world * 1000 * 2 / 0.125)


def test_single_rank_throughput():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_throughput(1, 256000, 3, 1500.0) == pytest.approx(256000 * 3 / 1.5)


def test_an_auxiliary_leg_that_fails_is_reported_in_the_line(capsys):
    sys.path.insert(0, ROOT)
    import bench

    assert bench.optional_leg("soc", lambda: {"value": 1.0}) == {"value": 1.0}

    def boom():
        raise RuntimeError("afqmc_soc_sweep_slice failed: -3")

    assert bench.optional_leg("soc", boom) == {"error": "RuntimeError: afqmc_soc_sweep_slice failed: -3"}
    assert "soc leg failed" in capsys.readouterr().err
