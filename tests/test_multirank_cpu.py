"""Replica aggregation of bench.py with two ranks on CPU (gloo): the barrier, the
max-over-ranks time and the sum of the ranks' flops (value = sum flops / max time)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    flops = [3.0e12, 5.0e12][rank]
    ms = [2000.0, 2500.0][rank]
    value, t_max = bench.aggregate(flops, ms, world)
    out[rank] = (value, t_max)
    dist.destroy_process_group()


def test_two_rank_aggregate():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        value, t_max = out[r]
        assert t_max == 2500.0
        assert abs(value - 8.0e12 / 2.5 / 1e9) < 1e-6
