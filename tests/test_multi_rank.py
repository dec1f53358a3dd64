"""Multi-process host logic of the benchmark (replicas, one lattice per rank):
max-over-ranks timing and whole-job throughput, on CPU with gloo, world
size 2.  The data path has no collective: ranks never exchange lattice data."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_max = bench.max_over_ranks(times[rank], dist)
    out.put((rank, t_max, bench.job_mlups(1000, 10, world, t_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [12.5, 40.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, v in res:
        assert t_max == 40.0
        assert v == pytest.approx(1000 * 10 * 2 / 0.040 / 1e6)


def test_single_process_aggregation():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    assert bench.max_over_ranks(3.0, None) == 3.0
    assert bench.job_mlups(4096 * 1024, 100, 1, 10.0) == pytest.approx(4096 * 1024 * 100 / 0.01 / 1e6)
