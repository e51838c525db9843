"""The sharded reductions on the library's kernels and NCCL, as a one-rank
group on one GPU (a rank that waits on no peer): each result equals the
plain call bit for bit, since the rank-ordered combination of one partial
returns it unchanged.  Runs in a spawned process so that the process group
does not outlive the test."""
import multiprocessing as mp
import os
import socket
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(port, q):
    try:
        sys.path.insert(0, ROOT)
        import torch
        import torch.distributed as dist
        import paper_cs_0603115_gb300 as ff
        from paper_cs_0603115_gb300 import dist as ffdist
        from paper_cs_0603115_gb300 import inputs
        torch.cuda.set_device(0)
        dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", world_size=1, rank=0,
                                device_id=torch.device("cuda", 0))
        g = inputs.ill_dot(1 << 20, 1e9, inputs.seed_for(2, 70), device="cuda")
        same = lambda a, b: bool(torch.equal(a.view(torch.int32), b.view(torch.int32)))
        ok = same(ffdist.sharded_dot(g.x, g.y), ff.dot(g.x, g.y))
        ok &= same(ffdist.sharded_sum(g.x), ff.sum(g.x))
        gi = inputs.gemv(300, 130, 3, inputs.seed_for(4, 140), device="cuda")
        ok &= same(ffdist.sharded_gemv_t(gi.A, gi.dY), ff.gemv_t(gi.A, gi.dY))
        torch.cuda.synchronize()
        dist.destroy_process_group()
        q.put(("ok" if ok else "mismatch", ""))
    except Exception as exc:  # reported to the parent
        q.put(("error", repr(exc)))


def test_sharded_reductions_one_rank_on_the_gpu():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_worker, args=(_free_port(), q))
    p.start()
    status, msg = q.get(timeout=300)
    p.join(timeout=60)
    assert status == "ok", msg
    assert p.exitcode == 0
