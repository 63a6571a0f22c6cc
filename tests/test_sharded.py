"""Row-block sharding of one product (rows of A and C across ranks, B broadcast
once, no reduction), on two and three gloo ranks on the CPU.

Each rank holds its block of A's rows and rank 0 alone holds B; the local
product of a rank is the CPU oracle here (on a GPU it is the library's
gf2_mul).  The stitched C on rank 0 must equal the oracle's product of the
whole matrices bit for bit, and every rank's block its own rows of it.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_0811_1714_gb300.sharded import row_blocks  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, m, l, n, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    import synth
    from paper_0811_1714_gb300.sharded import gf2_mul_sharded, row_blocks as blocks

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        r0, r1 = blocks(m, world)[rank]
        A = synth.random_packed(m, l, 41)
        B = synth.random_packed(l, n, 42)
        A_local = torch.from_numpy(np.ascontiguousarray(A[r0:r1]).view(np.int64))
        B_t = torch.from_numpy(B.view(np.int64).copy()) if rank == 0 else \
            torch.zeros(B.shape, dtype=torch.int64)            # only rank 0 holds B

        def local_mul(C, Ab, Bb):
            rows = Ab.shape[0]
            if rows:
                got = oracle.mul_packed(Ab.numpy().view(np.uint64), Bb.numpy().view(np.uint64), rows, l, n)
                C.copy_(torch.from_numpy(np.ascontiguousarray(got[:, :C.shape[1]]).view(np.int64)))

        C_local, C = gf2_mul_sharded(A_local, B_t, l, n, local_mul=local_mul)
        ref = oracle.mul_packed(A, B, m, l, n)
        W = synth.words_for(n)
        ok_local = np.array_equal(C_local.numpy().view(np.uint64)[:, :W], ref[r0:r1, :W])
        ok_b = np.array_equal(B_t.numpy().view(np.uint64), B)  # the broadcast reached every rank
        ok_full = True
        if rank == 0:
            ok_full = C is not None and np.array_equal(C.numpy().view(np.uint64)[:, :W], ref[:, :W])
        else:
            ok_full = C is None
        out[rank] = (ok_local, ok_b, ok_full)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,m,l,n", [(2, 300, 200, 150), (3, 130, 70, 65), (2, 40, 64, 64)])
def test_sharded_product_on_gloo_ranks(world, m, l, n):
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, m, l, n, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r] == (True, True, True), (r, out[r])


@pytest.mark.parametrize("m,world,align", [(0, 2, 64), (1, 3, 64), (1000, 4, 64), (32768, 8, 64), (130, 3, 1)])
def test_row_blocks_partition_the_rows(m, world, align):
    b = row_blocks(m, world, align)
    assert len(b) == world and b[0][0] == 0 and b[-1][1] == m
    for (a0, a1), (c0, c1) in zip(b, b[1:]):
        assert a1 == c0 and a0 <= a1
    for r0, r1 in b[:-1]:
        assert r0 % align == 0 and r1 % align == 0 or r1 == m
    sizes = [r1 - r0 for r0, r1 in b]
    assert max(sizes) - min(sizes) <= align
