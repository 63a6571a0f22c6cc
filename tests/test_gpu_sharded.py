"""The row-sharded product on the GPU: one NCCL rank (this run has one GPU),
the library's gf2_mul as the local product, compared with the CPU oracle.
The multi-rank partition, broadcast and stitching are covered on gloo ranks
in test_sharded.py."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _one_rank(port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import oracle
    import synth
    import paper_0811_1714_gb300 as g
    from paper_0811_1714_gb300.sharded import gf2_mul_sharded

    torch.cuda.set_device(0)
    g.build()
    dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % port, rank=0, world_size=1)
    try:
        m, l, n = 3000, 2000, 2500
        A = synth.random_packed(m, l, 51)
        B = synth.random_packed(l, n, 52)
        Ad = torch.from_numpy(A.view(np.int64)).cuda()
        Bd = torch.from_numpy(B.view(np.int64)).cuda()
        C_local, C = gf2_mul_sharded(Ad, Bd, l, n, options=g.opts(depth=1))
        torch.cuda.synchronize()
        ref = oracle.mul_packed(A, B, m, l, n)
        W = synth.words_for(n)
        got = C.cpu().numpy().view(np.uint64)[:, :W]
        out["ok"] = bool(np.array_equal(got, ref[:, :W])) and bool(torch.equal(C, C_local))
    finally:
        dist.destroy_process_group()


def test_sharded_product_on_one_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    p = ctx.Process(target=_one_rank, args=(_free_port(), out))
    p.start()
    p.join(300)
    assert p.exitcode == 0
    assert out.get("ok") is True
