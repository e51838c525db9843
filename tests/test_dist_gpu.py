"""The sharded reductions on the library's kernels: with NCCL as a one-rank
group on one GPU (a rank that waits on no peer), where each result equals
the plain call bit for bit, since the rank-ordered combination of one
partial returns it unchanged; and with two and three processes sharing the
GPU, each running its own kernels while the exchange of the float-float
partials runs over gloo on host copies, so that no kernel ever waits on
another process.  Runs in spawned processes so that the process groups do
not outlive the tests."""
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


def _gloo_worker(rank, world, port, q):
    """One of `world` processes sharing the GPU: the per-rank kernels and the
    rank-ordered combinations run on the GPU through the library; the
    exchange runs over gloo on host copies of the partials (no kernel of one
    rank waits on another rank)."""
    try:
        sys.path.insert(0, ROOT)
        import torch
        import torch.distributed as dist
        import paper_cs_0603115_gb300 as ff
        from paper_cs_0603115_gb300 import dist as ffdist
        from paper_cs_0603115_gb300 import inputs
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=world, rank=rank)
        dot_fn = lambda x, y: ff.dot(x.cuda(), y.cuda()).cpu()
        sum_fn = lambda v: ff.sum(v.cuda()).cpu()
        gt_fn = lambda A, dY: ff.gemv_t(A.cuda(), dY.cuda()).cpu()
        add_fn = lambda a, b: ff.add(a.cuda(), b.cuda()).cpu()
        n = 300007
        g = inputs.ill_dot(n, 1e9, inputs.seed_for(2, 71))
        lo, hi = ffdist.shard_range(n, rank, world)
        d = ffdist.sharded_dot(g.x[lo:hi], g.y[lo:hi], dot_fn=dot_fn, sum_fn=sum_fn)
        s = ffdist.sharded_sum(g.x[lo:hi], sum_fn=sum_fn)
        gi = inputs.gemv(301, 130, 3, inputs.seed_for(4, 141))
        r0, r1 = ffdist.shard_range(301, rank, world)
        dX = ffdist.sharded_gemv_t(gi.A[r0:r1].contiguous(), gi.dY[:, r0:r1].contiguous(), gemv_t_fn=gt_fn,
                                   add_fn=add_fn)
        torch.cuda.synchronize()
        dist.destroy_process_group()
        q.put((rank, d.numpy().tobytes(), s.numpy().tobytes(), dX.numpy().tobytes()))
    except Exception as exc:  # reported to the parent
        q.put((rank, "error", repr(exc), ""))


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_reductions_several_ranks_sharing_the_gpu(world):
    """Two and three processes on the one GPU: every rank holds the same
    bits, equal to the rank-ordered combination (done on the host with the
    oracle) of the shards' GPU results."""
    import numpy as np
    import oracle
    import paper_cs_0603115_gb300 as ff
    from paper_cs_0603115_gb300 import dist as ffdist
    from paper_cs_0603115_gb300 import inputs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(r[1] != "error" for r in res), [r[2] for r in res if r[1] == "error"]
    assert all(r[1:] == res[0][1:] for r in res)
    n = 300007
    g = inputs.ill_dot(n, 1e9, inputs.seed_for(2, 71))
    parts_d, parts_s = [], []
    for r in range(world):
        lo, hi = ffdist.shard_range(n, r, world)
        parts_d.append(ff.dot(g.x[lo:hi].cuda(), g.y[lo:hi].cuda()).cpu().numpy())
        parts_s.append(ff.sum(g.x[lo:hi].cuda()).cpu().numpy())
    np.testing.assert_array_equal(np.frombuffer(res[0][1], np.float32).view(np.uint32),
                                  oracle.ff_sum(np.stack(parts_d)).view(np.uint32))
    np.testing.assert_array_equal(np.frombuffer(res[0][2], np.float32).view(np.uint32),
                                  oracle.ff_sum(np.stack(parts_s)).view(np.uint32))
    gi = inputs.gemv(301, 130, 3, inputs.seed_for(4, 141))
    acc = None
    for r in range(world):
        r0, r1 = ffdist.shard_range(301, r, world)
        p = ff.gemv_t(gi.A[r0:r1].contiguous().cuda(), gi.dY[:, r0:r1].contiguous().cuda()).cpu().numpy()
        acc = p.reshape(-1, 2) if acc is None else oracle.add22(acc, p.reshape(-1, 2))
    np.testing.assert_array_equal(np.frombuffer(res[0][3], np.float32).view(np.uint32),
                                  acc.reshape(-1).view(np.uint32))
