"""The multi-GPU bench path's host logic on two gloo ranks (CPU): each rank
times its own batch, the job time is the slowest rank's, and the job rate is
all ranks' units over that time (weak scaling, no data-path collective)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(dist, 1.0 + 0.5 * rank)
    v = bench.whole_job_value(world, units_per_step=6 << 28, steps=10, elapsed_max=t)
    bench.barrier(dist)
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_two_rank_timing_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [1.5, 1.5]
    assert all(abs(r[2] - 2 * (6 << 28) * 10 / 1.5) < 1e-3 for r in res)


GEMV_T_SHAPES = [(12, 9, 3), (13, 10, 2), (7, 2, 1)]   # (m, n, k): n = 2 leaves a rank of 3 no column


def _shard_worker(rank, world, port, q):
    """Sharded dot, sum and GEMV adjoint on CPU ranks, with the oracle as the
    stand-in for the per-rank kernels (the exchange logic is what is under
    test)."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    from paper_cs_0603115_gb300 import dist as ffdist
    from paper_cs_0603115_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 10007
    g = inputs.ill_dot(n, 1e9, 4242)
    lo, hi = ffdist.shard_range(n, rank, world)
    dot_fn = lambda x, y: torch.from_numpy(oracle.ff_dot(x.numpy(), y.numpy()))
    sum_fn = lambda v: torch.from_numpy(oracle.ff_sum(v.numpy()))
    d = ffdist.sharded_dot(g.x[lo:hi], g.y[lo:hi], dot_fn=dot_fn, sum_fn=sum_fn)
    s = ffdist.sharded_sum(g.x[lo:hi], sum_fn=sum_fn)
    gt_fn = lambda A, dY: torch.from_numpy(oracle.gemv_t(A.numpy(), dY.numpy()))
    add_fn = lambda a, b: torch.from_numpy(oracle.add22(a.numpy().reshape(-1, 2), b.numpy().reshape(-1, 2)).reshape(a.shape))
    dXs = []
    for m, nn, k in GEMV_T_SHAPES:
        gi = inputs.gemv(m, nn, k, 77 + m)
        r0, r1 = ffdist.shard_range(m, rank, world)
        dX = ffdist.sharded_gemv_t(gi.A[r0:r1].contiguous(), gi.dY[:, r0:r1].contiguous(), gemv_t_fn=gt_fn,
                                   add_fn=add_fn)
        dXs.append(dX.numpy().tobytes())
    q.put((rank, d.numpy().tobytes(), s.numpy().tobytes(), *dXs))
    dist.destroy_process_group()


def _run_shards(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_reductions(world):
    import numpy as np
    import oracle
    from paper_cs_0603115_gb300 import dist as ffdist
    from paper_cs_0603115_gb300 import inputs
    res = _run_shards(world)
    # every rank holds the same bits
    assert all(r[1:] == res[0][1:] for r in res)
    # and they are the rank-ordered combination of the per-shard results
    n = 10007
    g = inputs.ill_dot(n, 1e9, 4242)
    x, y = g.x.numpy(), g.y.numpy()
    parts = []
    for r in range(world):
        lo, hi = ffdist.shard_range(n, r, world)
        parts.append(oracle.ff_dot(x[lo:hi], y[lo:hi]))
    want = oracle.ff_sum(np.stack(parts))
    got = np.frombuffer(res[0][1], np.float32)
    assert np.array_equal(got, want)
    _, _, A, E = oracle.exact_dot(x, y, got)
    assert abs(E) <= n * 2.0 ** -46 * A
    # GEMV adjoint: every column is the rank-ordered Add22 of the per-rank
    # partials (what an all-gather of whole partials followed by the same
    # combination on every rank gives), including a rank with no column
    for i, (m, nn, k) in enumerate(GEMV_T_SHAPES):
        gi = inputs.gemv(m, nn, k, 77 + m)
        dX = np.frombuffer(res[0][3 + i], np.float32).reshape(k, nn, 2)
        acc = None
        for r in range(world):
            r0, r1 = ffdist.shard_range(m, r, world)
            p = oracle.gemv_t(gi.A[r0:r1].numpy(), gi.dY[:, r0:r1].numpy()).reshape(-1, 2)
            acc = p if acc is None else oracle.add22(acc, p)
        np.testing.assert_array_equal(dX.view(np.uint32), acc.reshape(k, nn, 2).view(np.uint32))


def test_shard_ranges_cover_exactly():
    from paper_cs_0603115_gb300 import dist as ffdist
    for n in (0, 1, 7, 10007):
        for w in (1, 2, 3, 8):
            spans = [ffdist.shard_range(n, r, w) for r in range(w)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(h - l for l, h in spans) - min(h - l for l, h in spans) <= 1


def test_partition_instances_balances_bytes():
    from paper_cs_0603115_gb300 import dist as ffdist
    from paper_cs_0603115_gb300 import inputs
    lengths, kinds = inputs.batch_lengths(4096, inputs.seed_for(3, 0))
    nbytes = [16 * n if k == 0 else 24 * n for n, k in zip(lengths, kinds)]
    for world in (1, 2, 3, 8):
        parts = ffdist.partition_instances(nbytes, world)
        assert sorted(i for p in parts for i in p) == list(range(len(nbytes)))
        loads = [sum(nbytes[i] for i in p) for p in parts]
        assert max(loads) <= sum(nbytes) / world + max(nbytes)
        assert all(p == sorted(p) for p in parts)
    assert ffdist.partition_instances([], 4) == [[], [], [], []]
    assert ffdist.partition_instances([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]

