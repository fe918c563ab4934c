"""The replica path of bench.py (one independent replica per GPU, no data
exchange) on CPU: two gloo ranks agree on the slowest rank's step time and the
whole-job throughput counts every replica's work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, step_ms, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms_max = bench.max_over_ranks(step_ms[rank], dist)
        out[rank] = (ms_max, bench.whole_job_gflops(1e9, world, ms_max))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    step_ms = [0.25, 0.75]
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, step_ms, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 0.75
    # 2 replicas x 1 GFLOP each per 0.75 ms
    assert res[0][1] == pytest.approx(2.0 / 0.75e-3)


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(0.5) == 0.5
    assert bench.whole_job_gflops(4e9, 1, 2.0) == pytest.approx(2000.0)
