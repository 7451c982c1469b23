"""The N-GPU bench path runs independent replicas (one process per GPU, no
data-path collective): the whole-job time is the slowest rank's and the work
is the sum over ranks. Checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    assert bench.dist_env() == (rank, rank, world)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, u = bench.reduce_over_ranks(torch, dist, 1.5 + rank, 10 * (rank + 1), "cpu")
        out.put((rank, t, u))
    finally:
        dist.destroy_process_group()


def test_two_replicas_reduce_time_max_and_work_sum():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1:] for r in res] == [(2.5, 30.0), (2.5, 30.0)]


def test_one_process_is_its_own_total():
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    assert bench.reduce_over_ranks(torch, dist, 3.0, 7, "cpu") == (3.0, 7.0)
