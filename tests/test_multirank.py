"""Replica runs on several ranks, host logic only: two CPU ranks on the gloo
backend check that the bench's whole-job throughput sums the converged
solves of all ranks and divides by the slowest rank's timed region, as
`bench.py` does under torchrun with one GPU per rank (NCCL)."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r: 3 + r converged solves in (r + 1) seconds
    solves, ms, value = bench.job_throughput(3 + rank, 1000.0 * (rank + 1), dist)
    e2e = bench.world_reduce(0.5 * (rank + 1), dist, "cpu", "max")
    q.put((rank, solves, ms, value, e2e))
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_over_two_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, solves, ms, value, e2e in res:
        assert solves == 7.0 and ms == 2000.0 and value == 3.5 and e2e == 1.0, (rank, solves, ms, value, e2e)


def test_single_process_reduces_to_local_values():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(4, 2000.0) == (4, 2000.0, 2.0)
    assert bench.world_reduce(1.5) == 1.5
