"""The multi-rank benchmark path on CPU: world_size 2 over gloo.

bench.py --gpus N runs N independent replicas (the step needs no exchange
between ranks); its only collective is the max of the ranks' times, and the
job's throughput is all ranks' particle-steps over that max.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    slowest = bench.max_over_ranks(ms, dist, "cpu")
    value = bench.job_throughput(1000, world, 4, slowest * 1e-3)
    out[rank] = (slowest, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_throughput():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    slowest, value = res[0]
    assert slowest == 15.0
    assert value == pytest.approx(1000 * 2 * 4 / 0.015)


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(10, 1, 2, 0.5) == 40.0
