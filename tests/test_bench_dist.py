"""Host logic of the multi-GPU (replica) path of bench.py on CPU: two gloo ranks
aggregate their timed regions into whole-job throughput = summed units / max time."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = [2.0, 4.0][rank]
    units = [5, 5][rank]
    value, t, u = bench.aggregate(elapsed, units, dist, "cpu")
    q.put((rank, value, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t, u in out:
        assert t == 4.0 and u == 10.0
        assert value == pytest.approx(10.0 / 4.0)


def test_single_rank_aggregation():
    import bench
    assert bench.aggregate(2.0, 4) == (2.0, 2.0, 4)
