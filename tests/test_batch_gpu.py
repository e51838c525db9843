"""Batched dot / AXPY instances in one persistent launch (and its CUDA graph
and autotuner) against the oracle and against the plain per-instance calls.

AXPY instances must match the oracle bit for bit; dot instances must stay
within n 2^-46 sum|x_i y_i| of the exact value.  Lengths cover 0, 1, odd,
tile-sized and multi-tile instances; some instances start 8 bytes past a
16-byte boundary (scalar path).
"""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
from paper_cs_0603115_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = "cuda"


def same_bits(got, want):
    got = np.ascontiguousarray(got, np.float32)
    want = np.ascontiguousarray(want, np.float32)
    nan = np.isnan(got) & np.isnan(want)
    assert ((got.view(np.uint32) == want.view(np.uint32)) | nan).all()


def build_case(lengths, kinds, seed):
    from paper_cs_0603115_gb300 import batch
    specs, keep = [], []
    for i, (n, kind) in enumerate(zip(lengths, kinds)):
        # every fifth instance starts 8 bytes off a 16-byte boundary; of
        # those, every other one has its outputs off the boundary too (16-byte
        # access after one value), the others aligned outputs (8-byte access)
        mis = (i % 5 == 3)
        out_mis = mis and (i % 10 == 8)
        if kind == batch.DOT:
            g = inputs.ill_dot(max(n, 4), 1e8, seed + i)
            x, y = g.x[:n], g.y[:n]
        else:
            e = inputs.elementwise(n, seed + i)
            x, y = e.a, e.b
        xd = torch.empty((n + 1, 2), dtype=torch.float32, device=DEV)[int(mis):int(mis) + n]
        yd = torch.empty((n + 1, 2), dtype=torch.float32, device=DEV)[int(mis):int(mis) + n]
        xd.copy_(x)
        yd.copy_(y)
        alpha = inputs.scalar_ff(seed + 1000 + i)
        if kind == batch.DOT:
            out = torch.full((2,), float("nan"), dtype=torch.float32, device=DEV)
        else:
            out = torch.full((n + 1, 2), float("nan"), dtype=torch.float32,
                             device=DEV)[int(out_mis):int(out_mis) + n]
        if kind == batch.DOT_GRAD:
            out2 = torch.full((n + 1, 2), float("nan"), dtype=torch.float32, device=DEV)[int(mis):int(mis) + n]
            dout = alpha.to(DEV)
            specs.append((kind, xd, yd, out, None, out2, dout))
            keep.append((kind, x.numpy(), y.numpy(), alpha.numpy(), (out, out2)))
            continue
        specs.append((kind, xd, yd, out, (float(alpha[0]), float(alpha[1]))))
        keep.append((kind, x.numpy(), y.numpy(), alpha.numpy(), out))
    return specs, keep


def check(keep):
    from paper_cs_0603115_gb300 import batch
    for kind, x, y, alpha, out in keep:
        if kind == batch.DOT_GRAD:
            dx, dy = oracle.dot_backward(alpha, x, y)
            same_bits(out[0].cpu().numpy(), dx)
            same_bits(out[1].cpu().numpy(), dy)
            continue
        got = out.cpu().numpy()
        if kind == batch.AXPY:
            same_bits(got, oracle.axpy(alpha, x, y))
        else:
            _, _, A, E = oracle.exact_dot(x, y, got)
            assert abs(E) <= max(1, x.shape[0]) * 2.0 ** -46 * A


LENGTHS = [0, 1, 2, 3, 7, 100, 1000, 4095, 4096, 4097, 8191, 8192, 20001, 65536, 100003, 250000, 1, 5,
           33, 777, 3000, 12345, 54321, 99999]


@pytest.mark.parametrize("tune", [None, (128, 16, 0), (256, 64, 2), (512, 8, 4), (512, 64, 0), (256, 32, 0, 2), (128, 128, 2, 2)])
def test_batch_run_matches_oracle(tune):
    from paper_cs_0603115_gb300 import batch
    kinds = [batch.DOT if i % 2 else batch.AXPY for i in range(len(LENGTHS))]
    specs, keep = build_case(LENGTHS, kinds, 5000)
    plan = batch.BatchPlan(batch.make_instances(specs), tune=tune)
    plan.run()
    torch.cuda.synchronize()
    check(keep)
    # run again: counters were left at zero, partials are overwritten
    for _, _, _, _, out in keep:
        for t in (out if isinstance(out, tuple) else (out,)):
            t.fill_(float("nan"))
    plan.run()
    torch.cuda.synchronize()
    check(keep)
    plan.close()


@pytest.mark.parametrize("tune", [None, (256, 16, 0)])
def test_batch_with_dot_gradients(tune):
    from paper_cs_0603115_gb300 import batch
    kinds = [(batch.DOT, batch.AXPY, batch.DOT_GRAD)[i % 3] for i in range(len(LENGTHS))]
    specs, keep = build_case(LENGTHS, kinds, 6000)
    plan = batch.BatchPlan(batch.make_instances(specs), tune=tune).capture()
    plan.launch()
    torch.cuda.synchronize()
    check(keep)
    plan.close()


@pytest.mark.parametrize("tune", [None, (128, 16, 0)])
def test_batch_thousands_of_small_instances(tune):
    """3000 instances of 0 to 300 values, dot, AXPY and dot-gradient in
    turn: most are single-tile records and a block walks many of them.
    Every AXPY and gradient value bit for bit, every dot within its bound,
    on two runs (the second on the counters the first left at zero)."""
    from paper_cs_0603115_gb300 import batch
    rng = np.random.default_rng(77)
    lengths = [int(v) for v in rng.integers(0, 301, 3000)]
    kinds = [(batch.DOT, batch.AXPY, batch.DOT_GRAD)[i % 3] for i in range(len(lengths))]
    specs, keep = build_case(lengths, kinds, 9000)
    plan = batch.BatchPlan(batch.make_instances(specs), tune=tune)
    for _ in range(2):
        for _, _, _, _, out in keep:
            for t in (out if isinstance(out, tuple) else (out,)):
                t.fill_(float("nan"))
        plan.run()
        torch.cuda.synchronize()
        check(keep)
    plan.close()


def test_batch_graph_and_plain_agree():
    import paper_cs_0603115_gb300 as ff
    from paper_cs_0603115_gb300 import batch
    kinds = [batch.DOT if i % 3 else batch.AXPY for i in range(len(LENGTHS))]
    specs, keep = build_case(LENGTHS, kinds, 7000)
    plan = batch.BatchPlan(batch.make_instances(specs)).capture()
    plan.launch()
    plan.launch()
    torch.cuda.synchronize()
    check(keep)
    for kind, x, y, out, alpha in specs:
        if kind == batch.AXPY:
            same_bits(out.cpu().numpy(), ff.axpy(alpha, x, y).cpu().numpy())
        else:
            want = ff.dot(x, y).cpu().numpy()
            xs, ys = x.cpu().numpy(), y.cpu().numpy()
            _, _, A, _ = oracle.exact_dot(xs, ys)
            got = out.cpu().numpy()
            diff = abs((float(got[0]) - float(want[0])) + (float(got[1]) - float(want[1])))
            assert diff <= 2 * max(1, x.shape[0]) * 2.0 ** -46 * A
    plan.close()


def test_autotune_and_cache(tmp_path):
    from paper_cs_0603115_gb300 import batch
    kinds = [batch.DOT if i % 2 else batch.AXPY for i in range(len(LENGTHS))]
    specs, keep = build_case(LENGTHS, kinds, 9000)
    inst = batch.make_instances(specs)
    cache = str(tmp_path / "tune.json")
    tune, ms = batch.autotune(inst, reps=1, cache_path=cache)
    assert tune in batch.candidates()
    assert ms is not None and ms > 0
    tune2, ms2 = batch.autotune(inst, reps=1, cache_path=cache)
    assert tune2 == tune and ms2 is None
    plan = batch.BatchPlan(inst, tune=tune)
    plan.run()
    torch.cuda.synchronize()
    check(keep)
    plan.close()


def test_batch_errors():
    from paper_cs_0603115_gb300 import _lib, batch
    x = torch.zeros((10, 2), device=DEV)
    out = torch.zeros((10, 2), device=DEV)
    inst = batch.make_instances([(batch.AXPY, x, x, out, (1.0, 0.0))])
    L = _lib.load()
    with pytest.raises(ValueError):                 # the wrapper refuses an unknown kind
        batch.make_instances([(7, x, x, out, None)])
    bad = batch.make_instances([(batch.AXPY, x, x, out, (1.0, 0.0))])
    bad[0].kind = 7                                 # and so does the C ABI, given the raw record
    h = ctypes.c_void_p()
    assert L.ff_batch_plan_create(bad, 1, None, ctypes.byref(h)) == 1
    t = _lib.ff_tune(256, 3, 0)     # unsupported pairs_per_thread
    assert L.ff_batch_plan_create(inst, 1, ctypes.byref(t), ctypes.byref(h)) == 1
    plan = batch.BatchPlan(inst)
    assert L.ff_batch_run(plan.handle, plan.ws.data_ptr(), 8, None) == 2   # workspace too small
    plan.close()


@pytest.mark.parametrize("tune", [None, (128, 16, 0), (512, 64, 2), (256, 32, 0, 2)])
def test_batch_gemv_instances(tune):
    """GEMV instances of uneven shapes (rows become dot records) mixed with
    dots and AXPYs: every row within the dot bound of the exact value, and
    equal to the plain ff_gemv within twice the bound."""
    import paper_cs_0603115_gb300 as ff
    from paper_cs_0603115_gb300 import batch
    shapes = [(1, 1), (3, 1000), (17, 4097), (64, 9), (0, 5), (5, 0), (40, 20001), (3, 70001), (2, 65536)]
    specs, keep = [], []
    for i, (m, n) in enumerate(shapes):
        gi = inputs.gemv(m, n, 1, inputs.seed_for(4, 70 + i))
        A, x = gi.A.to(DEV), gi.X[0].to(DEV).contiguous()
        out = torch.full((m, 2), float("nan"), dtype=torch.float32, device=DEV)
        specs.append((batch.GEMV, A, x, out, None))
        keep.append((gi.A.numpy(), gi.X[0].numpy(), A, x, out))
    dspecs, dkeep = build_case([100, 7, 4097], [batch.DOT, batch.AXPY, batch.DOT], 8000)
    plan = batch.BatchPlan(batch.make_instances(specs + dspecs), tune=tune).capture()
    plan.launch()
    torch.cuda.synchronize()
    check(dkeep)
    for An, xn, A, x, out in keep:
        got = out.cpu().numpy()
        m, n = An.shape[0], An.shape[1]
        if m and n:
            plain = ff.gemv(A, x.reshape(1, n, 2))[0].cpu().numpy()
        for r in range(m):
            _, _, Aabs, E = oracle.exact_dot(An[r], xn, got[r])
            assert abs(E) <= max(1, n) * 2.0 ** -46 * Aabs
            if n:
                d = abs((float(got[r, 0]) - float(plain[r, 0])) + (float(got[r, 1]) - float(plain[r, 1])))
                assert d <= 2 * max(1, n) * 2.0 ** -46 * Aabs
            else:
                assert got[r, 0] == 0 and got[r, 1] == 0
    plan.close()


@pytest.mark.parametrize("tune", [None, (128, 16, 0), (512, 64, 2), (256, 32, 0, 2)])
def test_batch_gemv_only_plan_bitexact(tune):
    """A plan made only of GEMV rows (its own kernel: tiles sorted by cost,
    taken from an atomic counter): every row bit for bit equal to the replay
    of the eight-lane row order, on a plain run and on two graph replays."""
    from paper_cs_0603115_gb300 import batch
    import replay
    shapes = [(1, 1), (3, 1000), (17, 4097), (64, 9), (0, 5), (5, 0), (33, 64), (7, 4096), (129, 32),
              (2, 65536), (300, 3)]
    specs, keep = [], []
    for i, (m, n) in enumerate(shapes):
        gi = inputs.gemv(m, n, 1, inputs.seed_for(4, 110 + i))
        A, x = gi.A.to(DEV), gi.X[0].to(DEV).contiguous()
        out = torch.full((m, 2), float("nan"), dtype=torch.float32, device=DEV)
        specs.append((batch.GEMV, A, x, out, None))
        keep.append((gi.A.numpy(), gi.X[0].numpy(), out, n % 2 == 0))
    plan = batch.BatchPlan(batch.make_instances(specs), tune=tune)
    plan.run()
    torch.cuda.synchronize()
    want = [replay.gemv_rows8_replay(An, xn, vec) for An, xn, _, vec in keep]
    for (An, xn, out, vec), w in zip(keep, want):
        same_bits(out.cpu().numpy(), w)
        out.fill_(float("nan"))
    plan.capture()
    for _ in range(2):
        plan.launch()
        torch.cuda.synchronize()
        for (An, xn, out, vec), w in zip(keep, want):
            same_bits(out.cpu().numpy(), w)
            out.fill_(float("nan"))
    plan.close()


@pytest.mark.parametrize("tune", [(256, 32, 0, 4), (128, 16, 0, 2), (512, 64, 2, 4), (256, 128, 4, 2)])
def test_batch_dot_bitexact_vs_order_replay(tune):
    """DOT instances of a batched plan, aligned (16-byte access), both
    arrays 8 bytes off a 16-byte boundary (a one-value head, then 16-byte
    access) and of mixed alignment (8-byte access), one tile and many: bit
    for bit against the replay of the kernel's tile, thread and block order
    for this tune."""
    from paper_cs_0603115_gb300 import batch
    import replay
    lengths = [0, 1, 7, 8191, 8192, 8193, 100001, 33, 2, 4097, 65537, 3]
    g = inputs.ill_dot(sum(lengths) + 4 * len(lengths) + 4, 1e8, inputs.seed_for(3, 60))
    X, Y = g.x.to(DEV), g.y.to(DEV)
    D = torch.full((len(lengths), 2), float("nan"), device=DEV)
    specs, keep, o = [], [], 0
    for i, n in enumerate(lengths):
        # instance i % 3: 0 both aligned (16-byte access), 1 both 8 bytes
        # past a boundary (one value, then 16-byte access), 2 only y past a
        # boundary (8-byte access)
        offx = o + (i % 3 == 1)
        offy = o + (i % 3 >= 1)
        xs, ys = X[offx:offx + n], Y[offy:offy + n]
        specs.append((batch.DOT, xs, ys, D[i], None))
        keep.append((xs.cpu().numpy(), ys.cpu().numpy(), (1, 2, 0)[i % 3]))
        o = max(offx, offy) + n + 2
        o += o % 2
    plan = batch.BatchPlan(batch.make_instances(specs), tune=tune)
    plan.run()
    torch.cuda.synchronize()
    got = D.cpu().numpy()
    for i, (xn, yn, vec) in enumerate(keep):
        same_bits(got[i], replay.batch_dot_replay(xn, yn, tune[0], tune[1], vec))
    plan.close()

