"""bench.py's multi-rank path on CPU: replicas report the slowest rank's time and
the units processed by every rank (gloo, world size 2)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    ms, units = bench.reduce_over_ranks(100.0 + 50.0 * rank, 1000 * (rank + 1))
    out[rank] = (ms, units)
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == (150.0, 3000.0)
    assert out[1] == (150.0, 3000.0)


def test_single_process_passthrough():
    import bench
    assert bench.reduce_over_ranks(12.5, 7) == (12.5, 7)
