"""The multi-GPU form is N independent replicas: each rank sorts its own
arrays, and the bench reports the whole job's keys over the slowest rank's
time. The cross-rank step is checked here with two CPU ranks on gloo."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]
    value, ms = bench.replica_throughput(local_ms, 10**9, world, torch.device("cpu"))
    out.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in res:
        assert ms == 250.0                       # max over ranks
        assert abs(value - 2 * 10**9 / 0.25 / 1e9) < 1e-9   # both ranks' keys / slowest time


def test_single_rank_needs_no_collective():
    import bench
    value, ms = bench.replica_throughput(50.0, 10**8, 1, None)
    assert ms == 50.0 and abs(value - 2.0) < 1e-12
