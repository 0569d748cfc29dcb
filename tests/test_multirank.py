"""The N > 1 path of bench.py on CPU: two gloo ranks, the whole-job value is the sum of the ranks'
zone updates over the slowest rank's time (independent blocks per rank, no data-path collective)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r: 1000 * (r + 1) zones in 100 * (r + 1) ms per step
    value, ms, n = bench.aggregate(100.0 * (rank + 1), 1000 * (rank + 1), steps=3, dist=dist, device="cpu")
    out.put((rank, value, ms, n))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms, n in res:
        assert n == 2
        assert ms == 200.0  # the slowest rank
        assert value == pytest.approx(3000 * 3 / 0.2)  # all zones over the slowest time


def test_single_process_aggregation():
    import bench
    value, ms, n = bench.aggregate(50.0, 500, steps=4)
    assert n == 1 and value == pytest.approx(500 * 4 / 0.05)
