"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, nothing exchanged on the
data path) combine their timings through bench.reduce_over_ranks -- the job is as slow as
its slowest rank -- and the reference arm's non-zero ranks exit without work."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [10.0 + rank, 20.0 - rank]           # rank 1 slower in the first, faster in the second
    rates = [5.0 - rank]
    t, r = bench.reduce_over_ranks(torch, times, rates, world, "cpu")
    out[rank] = (t, r)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == ([11.0, 20.0], [4.0])


def test_single_rank_is_identity():
    import torch
    import bench
    assert bench.reduce_over_ranks(torch, [3.0, 4.0], [2.0], 1, "cpu") == ([3.0, 4.0], [2.0])


def test_reference_arm_other_ranks_do_nothing(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus = 1, 3, 2
    assert bench.run_reference(A()) == 0
