"""World-size-2 gloo run of bench.py's cross-rank timing logic (CPU only).

Each rank runs an independent job (weak scaling, no data-path collective); the
only exchange is the max over ranks of the step time, on a gloo group.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = dist.new_group(backend="gloo")
    ms = [120.0, 150.0][rank]                      # rank 1 is the slow one
    m = bench.reduce_max(ms, dist, g)
    v = bench.weak_scaling_value(1.0e9, world, m)
    out.put((rank, m, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == 150.0                           # every rank sees the slowest step
        assert abs(v - 2 * 1.0e9 / 0.150) < 1e-3    # units of both ranks / slowest time


def test_single_rank_identity():
    import bench
    assert bench.reduce_max(7.5) == 7.5
    assert bench.weak_scaling_value(10.0, 1, 1000.0) == 10.0
