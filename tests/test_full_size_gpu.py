"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times, on outputs the oracle can check one by one: the batched workload of
4096 dot and AXPY instances (3.7e9 values, the autotuner's launch shape) and
the GEMV family on the 32768 x 32768 matrix, and the adjoint of the 2^26-value
dot.  The elementwise operators and the reductions at full size are covered
in test_parity_gpu.py and test_compensated_gpu.py, the 4096^3 GEMM in
test_gemm_gpu.py."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_cs_0603115_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = "cuda"

if torch.cuda.is_available():
    import paper_cs_0603115_gb300 as ff


def same_bits(got, want):
    got = np.ascontiguousarray(got, np.float32)
    want = np.ascontiguousarray(want, np.float32)
    assert got.shape == want.shape
    nan = np.isnan(got) & np.isnan(want)
    assert ((got.view(np.uint32) == want.view(np.uint32)) | nan).all()


def _sample(idx, count, rng):
    """`count` indices of `idx` (a list ordered by length), always with the
    shortest and the longest."""
    pick = set(rng.choice(len(idx), size=min(count, len(idx)) - 2, replace=False).tolist()) | {0, len(idx) - 1}
    return [idx[p] for p in sorted(pick)]


def test_batched_4096_instances_full_size_sampled():
    """bench.py's batched workload (4096 instances, lengths log-uniform over
    1e2..1e7, dots at cond 1e8 and AXPY with 10% cancelling pairs, every
    instance at a 16-byte boundary) run once with the launch shape the
    autotuner picks: 24 sampled AXPY instances bit for bit against the
    oracle; 24 sampled dots within n 2^-46 sum |x_i y_i| of the exact value
    and, up to 2e5 values, bit for bit against the replay of the batched
    tile, thread and block order."""
    import replay
    from paper_cs_0603115_gb300 import batch
    lengths, kinds = inputs.batch_lengths(4096, inputs.seed_for(3, 0))
    offs, o = [], 0
    for n in lengths:
        offs.append(o)
        o += n + (n & 1)
    X = torch.empty((o, 2), dtype=torch.float32, device=DEV)
    Y = torch.empty((o, 2), dtype=torch.float32, device=DEV)
    Z = torch.full((o, 2), float("nan"), dtype=torch.float32, device=DEV)
    D = torch.full((4096, 2), float("nan"), dtype=torch.float32, device=DEV)
    alphas = [tuple(float(v) for v in inputs.scalar_ff(inputs.seed_for(3, 3) + i)) for i in range(4096)]
    sl = [slice(offs[i], offs[i] + lengths[i]) for i in range(4096)]
    for i, (n, kind) in enumerate(zip(lengths, kinds)):
        if kind == batch.DOT:
            g = inputs.ill_dot(n, 1e8, inputs.seed_for(3, 1) + 7 * i, device=DEV)
            X[sl[i]].copy_(g.x)
            Y[sl[i]].copy_(g.y)
        else:
            e = inputs.elementwise(n, inputs.seed_for(3, 2) + 7 * i, device=DEV)
            X[sl[i]].copy_(e.a)
            Y[sl[i]].copy_(e.b)
    specs = [(k, X[sl[i]], Y[sl[i]], D[i] if k == batch.DOT else Z[sl[i]], alphas[i]) for i, k in enumerate(kinds)]
    inst = batch.make_instances(specs)
    tune, _ = batch.autotune(inst, reps=1, cache_path=None)
    for t in (Z, D):
        t.fill_(float("nan"))   # the autotuner's runs wrote them
    plan = batch.BatchPlan(inst, tune=tune)
    plan.run()
    torch.cuda.synchronize()
    block, ppt = plan.tune[0], plan.tune[1]
    rng = np.random.default_rng(11)
    by_len = sorted(range(4096), key=lambda i: lengths[i])
    for i in _sample([j for j in by_len if kinds[j] == batch.AXPY], 24, rng):
        x, y = X[sl[i]].cpu().numpy(), Y[sl[i]].cpu().numpy()
        same_bits(Z[sl[i]].cpu().numpy(), oracle.axpy(np.array(alphas[i], np.float32), x, y))
    for i in _sample([j for j in by_len if kinds[j] == batch.DOT], 24, rng):
        x, y = X[sl[i]].cpu().numpy(), Y[sl[i]].cpu().numpy()
        got = D[i].cpu().numpy()
        _, _, a_abs, err = oracle.exact_dot(x, y, got)
        assert abs(err) <= lengths[i] * 2.0 ** -46 * a_abs
        if lengths[i] <= 200000:
            same_bits(got, replay.batch_dot_replay(x, y, block, ppt, 1))
    plan.close()
    del X, Y, Z, D
    torch.cuda.empty_cache()


def test_gemv_family_full_size_sampled():
    """The 32768 x 32768 matrix (8 GiB) of bench.py's GEMV sweep: with k = 3,
    Y = A X on 16 sampled rows and dX = A^T dY on 16 sampled columns bit for
    bit against the replays of their orders (the adjoint's row blocks read
    from ff_gemv_t_launch_shape at this size); the weight gradient
    dA = dY X^T with k = 3 (one pass) and k = 20 (two passes) on a 16 x 16
    sample of elements bit for bit against the oracle."""
    import replay
    from paper_cs_0603115_gb300 import _lib
    M = N = 32768
    gi = inputs.gemv(M, N, 20, inputs.seed_for(4, 180), device=DEV)
    A = gi.A
    rng = np.random.default_rng(12)
    rows = sorted(set(rng.choice(M, 14, replace=False).tolist()) | {0, M - 1})
    cols = sorted(set(rng.choice(N, 14, replace=False).tolist()) | {0, N - 1})
    X3, dY3 = gi.X[:3].contiguous(), gi.dY[:3].contiguous()
    Y = ff.gemv(A, X3)
    dX = ff.gemv_t(A, dY3)
    torch.cuda.synchronize()
    same_bits(Y[:, rows].cpu().numpy(), replay.gemv_warp_replay(A[rows].cpu().numpy(), X3.cpu().numpy(), vec=True))
    nrb, vec = ctypes.c_int64(), ctypes.c_int()
    _lib.call("ff_gemv_t_launch_shape", A.data_ptr(), M, N, N, 3, ctypes.byref(nrb), ctypes.byref(vec))
    assert vec.value == 1
    same_bits(dX[:, cols].cpu().numpy(),
              replay.gemv_t_replay(A[:, cols].cpu().numpy(), dY3.cpu().numpy(), nrb.value))
    del Y, dX
    dA = torch.empty_like(A)
    Xc, dYr = gi.X[:, cols].cpu().numpy(), gi.dY[:, rows].cpu().numpy()
    for k in (3, 20):
        dA.fill_(float("nan"))
        ff.gemv_dA(gi.dY[:k].contiguous(), gi.X[:k].contiguous(), out=dA)
        torch.cuda.synchronize()
        got = dA[rows][:, cols].cpu().numpy()
        same_bits(got, oracle.gemv_dA(np.ascontiguousarray(dYr[:k]), np.ascontiguousarray(Xc[:k])))
    del dA, gi, A
    torch.cuda.empty_cache()


def test_dot_adjoint_full_size():
    """The dot of 2^26 values at cond 1e12 (bench.py's workload) through the
    autograd function: dx = Mul22(dout, y) and dy = Mul22(dout, x) bit for
    bit against the oracle on 2^20 sampled indices plus both ends, and two
    sampled entries of dx against central finite differences of the exact
    dot (binary128 superaccumulator over all 2^26 terms)."""
    import math
    n = 1 << 26
    g = inputs.ill_dot(n, 1e12, inputs.seed_for(2, 12), device=DEV)
    dout = inputs.scalar_ff(321)
    x = g.x.clone().requires_grad_(True)
    y = g.y.clone().requires_grad_(True)
    ff.ffdot(x, y).backward(dout.to(DEV))
    gen = torch.Generator().manual_seed(99)
    idx = torch.cat([torch.arange(1024), torch.randint(0, n, (1 << 20,), generator=gen),
                     torch.arange(n - 1024, n)]).to(DEV)
    xs, ys = g.x[idx].cpu().numpy(), g.y[idx].cpu().numpy()
    dx_want, dy_want = oracle.dot_backward(dout.numpy(), xs, ys)
    same_bits(x.grad[idx].cpu().numpy(), dx_want)
    same_bits(y.grad[idx].cpu().numpy(), dy_want)
    xn, yn = g.x.cpu().numpy(), g.y.cpu().numpy()
    dval = float(dout[0]) + float(dout[1])
    rng = np.random.default_rng(7)
    for i in rng.choice(n, size=2, replace=False):
        hi = float(xn[i, 0])
        h = 2.0 ** (math.floor(math.log2(abs(hi))) - 10)
        old = xn[i, 0]
        xn[i, 0] = np.float32(hi + h)
        sp = oracle.exact_dot(xn, yn)
        xn[i, 0] = np.float32(hi - h)
        sm = oracle.exact_dot(xn, yn)
        xn[i, 0] = old
        fd = dval * ((sp[0] - sm[0]) + (sp[1] - sm[1])) / (2.0 * h)
        got = float(x.grad[i, 0]) + float(x.grad[i, 1])
        assert abs(got - fd) <= (2.0 ** -44 + 2.0 ** -50) * abs(fd)
    del g, x, y
    torch.cuda.empty_cache()


def test_gemv_family_beyond_2_31_elements():
    """A 65600 x 32768 matrix (2.15e9 elements, past 2^31, 17 GB): every
    offset into A, dA and the adjoint's workspace needs 64 bits.  Rows and
    columns sampled near both ends: Y and dX bit for bit against the
    replays of their orders, dA (k = 1) against the oracle."""
    import replay
    from paper_cs_0603115_gb300 import _lib
    M, N = 65600, 32768
    assert M * N > 2 ** 31
    gi = inputs.gemv(M, N, 1, inputs.seed_for(4, 190), device=DEV)
    A = gi.A
    rows = [0, 1, 32767, 32768, 65535, 65536, M - 2, M - 1]
    cols = [0, 1, 16383, 16384, N - 2, N - 1]
    Y = ff.gemv(A, gi.X)
    dX = ff.gemv_t(A, gi.dY)
    torch.cuda.synchronize()
    same_bits(Y[:, rows].cpu().numpy(), replay.gemv_warp_replay(A[rows].cpu().numpy(), gi.X.cpu().numpy(), vec=True))
    nrb, vec = ctypes.c_int64(), ctypes.c_int()
    _lib.call("ff_gemv_t_launch_shape", A.data_ptr(), M, N, N, 1, ctypes.byref(nrb), ctypes.byref(vec))
    same_bits(dX[:, cols].cpu().numpy(),
              replay.gemv_t_replay(A[:, cols].cpu().numpy(), gi.dY.cpu().numpy(), nrb.value))
    del Y, dX
    dA = torch.empty_like(A)
    ff.gemv_dA(gi.dY, gi.X, out=dA)
    torch.cuda.synchronize()
    got = dA[rows][:, cols].cpu().numpy()
    same_bits(got, oracle.gemv_dA(np.ascontiguousarray(gi.dY[:, rows].cpu().numpy()),
                                  np.ascontiguousarray(gi.X[:, cols].cpu().numpy())))
    del dA, gi, A
    torch.cuda.empty_cache()


def test_gemm_beyond_2_31_elements():
    """C = A B of 65600 x 32768 (2.15e9 elements, past 2^31) with k = 3:
    rows sampled near both ends bit for bit against the oracle's in-order
    loop (64-bit offsets into C)."""
    M, N, K = 65600, 32768, 3
    gen = torch.Generator(device=DEV).manual_seed(inputs.seed_for(6, 190))
    A = inputs.to_ff(inputs.loguniform_f64(M * K, gen, DEV)).reshape(M, K, 2)
    B = inputs.to_ff(inputs.loguniform_f64(K * N, gen, DEV)).reshape(K, N, 2)
    C = ff.gemm(A, B)
    torch.cuda.synchronize()
    rows = [0, 1, 32767, 32768, 65535, 65536, M - 1]
    got = C[rows].cpu().numpy()
    want = oracle.gemm(np.ascontiguousarray(A[rows].cpu().numpy()), B.cpu().numpy())
    same_bits(got, want)
    del C, A, B
    torch.cuda.empty_cache()


def test_batched_instance_beyond_2_31_values():
    """One AXPY instance of 2^31 + 5 values (17 GB per array) next to a small
    dot instance in one batched plan: the values near both ends and around
    2^31 bit for bit against the oracle (64-bit tile offsets)."""
    from paper_cs_0603115_gb300 import batch
    n = (1 << 31) + 5
    gen = torch.Generator(device=DEV).manual_seed(inputs.seed_for(3, 190))
    x = inputs.to_ff(inputs.loguniform_f64(n, gen, DEV))
    y = inputs.to_ff(inputs.loguniform_f64(n, gen, DEV))
    z = torch.empty_like(x)
    d = torch.empty(2, dtype=torch.float32, device=DEV)
    alpha = (1.25, 2.0 ** -30)
    plan = batch.BatchPlan(batch.make_instances([(batch.AXPY, x, y, z, alpha),
                                                 (batch.DOT, x[:1000], y[:1000], d, None)]))
    plan.run()
    torch.cuda.synchronize()
    # contiguous slices copied to the host (no gather kernel: PyTorch's
    # index kernel asserted on an index tensor into these 2^31 + 5 rows)
    spans = [(0, 4096), ((1 << 31) - 4096, (1 << 31) + 4096), (n - 4096, n)]
    take = lambda t: np.concatenate([t[lo:hi].cpu().numpy() for lo, hi in spans])
    same_bits(take(z), oracle.axpy(np.array(alpha, np.float32), take(x), take(y)))
    _, _, a_abs, err = oracle.exact_dot(x[:1000].cpu().numpy(), y[:1000].cpu().numpy(), d.cpu().numpy())
    assert abs(err) <= 1000 * 2.0 ** -46 * a_abs
    plan.close()
    del x, y, z
    torch.cuda.empty_cache()
