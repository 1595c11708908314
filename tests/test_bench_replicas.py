"""The N > 1 path of bench.py ("replicas only": independent copies of the workload, no data-path
collective) on CPU with two gloo ranks: the job's time is the slowest rank's, the throughput the
units of all ranks over that time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.replica_time(1.0 + rank, dist, "cpu")  # rank 1 is the slower replica
    value = bench.replica_throughput(340e6, world, ms)
    out.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in got:
        assert ms == pytest.approx(2.0)                       # max over ranks
        assert value == pytest.approx(2 * 340e6 / 2.0e-3)      # both ranks' bytes over the job time


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.replica_time(1.5, None, "cpu") == 1.5
    assert bench.replica_throughput(10.0, 1, 2.0) == pytest.approx(5000.0)
