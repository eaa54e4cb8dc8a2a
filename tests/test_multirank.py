"""The multi-rank path of the bench on CPU: world size 2 over gloo.

The method's units (fields) are independent, so ranks are replicas: each
compresses its own field and the only exchange is the max of the timings.
These tests run that exchange and the job-throughput arithmetic on two
processes, with no GPU.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r's times: the slowest rank decides every entry
        mine = [10.0 + rank, 3.0 - rank, 7.5 * (rank + 1)]
        got = bench.max_over_ranks(mine, dist)
        dist.barrier()
        q.put((rank, got, bench.replica_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_seeds():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get() for _ in range(2))
    for _, got, _ in res:
        assert got == [11.0, 3.0, 15.0]
    # each replica compresses its own field
    assert res[0][2] != res[1][2]


def test_job_throughput_arithmetic():
    import bench
    # two replicas of 512^3 float32 in 4.74 ms: the whole job's input bytes
    n = 512 ** 3
    assert bench.job_gbps(2, n, 4.74e-3) == pytest.approx(2 * 4 * n / 4.74e-3 / 1e9)
    assert bench.job_gbps(1, n, 1.0) == pytest.approx(4 * n / 1e9)
    assert bench.max_over_ranks([1.5, 2.5], None) == [1.5, 2.5]
