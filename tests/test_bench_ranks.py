"""The multi-rank path of bench.py on the CPU: two ranks over gloo (127.0.0.1).  Each rank solves
its own replica system; the job's time is the slowest rank's, and seconds per system divide it by
the systems all ranks processed."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 * (rank + 1)                        # rank 1 is the slow one
    out.put((rank, bench.max_over_ranks(ms, dist, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert results == [(0, 200.0), (1, 200.0)]


def test_seconds_per_system_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.seconds_per_system(600.0, 3, 2) == pytest.approx(0.1)
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
