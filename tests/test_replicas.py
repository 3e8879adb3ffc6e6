"""Multi-GPU runs are independent replicas (the method is single-domain): the
benchmark's only cross-rank step is the max-over-ranks time. Two gloo ranks
on CPU exercise that path."""
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


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    value, t = bench.replica_throughput(100.0 * (rank + 1), 1000, 10, ws)
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        # slowest rank: 200 ms for 10 steps of 1000 nodes on each of 2 ranks
        for r in range(ws):
            value, t = out[r]
            assert t == 200.0
            assert abs(value - 1000 * 10 * 2 / 0.2 / 1e6) < 1e-12


def test_replica_throughput_single_rank():
    import bench
    value, t = bench.replica_throughput(50.0, 2000, 5, 1)
    assert t == 50.0 and abs(value - 2000 * 5 / 0.05 / 1e6) < 1e-12
