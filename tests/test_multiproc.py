"""The multi-rank timing of bench.py over two gloo ranks on CPU (no GPU):
whole-job value = bit operations of all ranks over the slowest rank's time."""
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


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        ms, ops, value = bench.aggregate(10.0 * (rank + 1), 1e12 * (rank + 1))
        dist.barrier()
        out[rank] = (ms, ops, value)
    finally:
        dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        ms, ops, value = out[r]
        assert ms == 20.0                        # the slowest rank
        assert ops == 3e12                       # the work of both ranks
        assert abs(value - 3e12 / 0.02) < 1.0


def test_aggregate_single_process():
    import bench
    ms, ops, value = bench.aggregate(5.0, 1e9)
    assert (ms, ops) == (5.0, 1e9) and abs(value - 2e11) < 1e-3
