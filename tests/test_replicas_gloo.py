"""The N > 1 path of bench.py on CPU: replicas (one independent solve stream
per rank, no collective on the data path) report the whole-job throughput as
all ranks' units over the slowest rank's timed region (max over ranks by an
all-reduce).  Two gloo ranks on 127.0.0.1."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [800.0, 1000.0][rank]  # rank 1 is the slow replica
    ms, value = bench.replica_throughput(dist, world, 10, local_ms, "cpu")
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, value in out:
        assert ms == 1000.0                       # the slowest replica's time on every rank
        assert value == pytest.approx(20 / 1.0)   # 2 ranks x 10 units in 1 s


def test_replica_throughput_single_process():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.replica_throughput(None, 1, 5, 500.0, "cpu") == (500.0, 10.0)
