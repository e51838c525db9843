"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Elementwise operators must match the oracle bit for bit (NaN == NaN);
reductions must match a replay of their documented order bit for bit and stay
within n 2^-46 sum|x_i y_i| of the exact value; GEMV rows stay within the
same bound.  Sizes span several tiles and ragged tails; edge cases cover
empty input, one to three elements, misaligned and mixed-alignment arrays,
in-place operation, signed zeros, subnormals and specials.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_cs_0603115_gb300 import inputs

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_cs_0603115_gb300 as ff
    from paper_cs_0603115_gb300 import _lib

DEV = "cuda"
N0 = 1 << 20


def same_bits(got, want):
    got = np.ascontiguousarray(got, np.float32)
    want = np.ascontiguousarray(want, np.float32)
    assert got.shape == want.shape
    nan = np.isnan(got) & np.isnan(want)
    eq = (got.view(np.uint32) == want.view(np.uint32)) | nan
    if not eq.all():
        bad = np.argwhere(~eq)[:5]
        raise AssertionError(f"{(~eq).sum()} mismatches, first at {bad.tolist()}: "
                             f"got {got[tuple(bad[0])]} want {want[tuple(bad[0])]}")


@pytest.fixture(scope="module")
def cfg0():
    e = inputs.elementwise(N0 + 3, inputs.seed_for(0, 0))
    return e


def gpu(t):
    return t.to(DEV)


# ---------------------------------------------------------------------------
# elementwise, bit-exact
# ---------------------------------------------------------------------------

def test_add12_mul12_bitexact(cfg0):
    ab = cfg0.ab
    same_bits(ff.add12(gpu(ab)).cpu().numpy(), oracle.add12(ab.numpy()))
    same_bits(ff.mul12(gpu(ab)).cpu().numpy(), oracle.mul12(ab.numpy()))


@pytest.mark.parametrize("op", ["add", "mul", "div"])
def test_binary_ops_bitexact(cfg0, op):
    a, b = cfg0.a, cfg0.b
    got = getattr(ff, op)(gpu(a), gpu(b)).cpu().numpy()
    want = {"add": oracle.add22, "mul": oracle.mul22, "div": oracle.div22}[op](a.numpy(), b.numpy())
    same_bits(got, want)


def test_sqrt_bitexact(cfg0):
    a = cfg0.a_sqrt
    same_bits(ff.sqrt(gpu(a)).cpu().numpy(), oracle.sqrt22(a.numpy()))


def test_axpy_and_dot_backward_bitexact(cfg0):
    a, b = cfg0.a, cfg0.b
    alpha = inputs.scalar_ff(99).numpy()
    same_bits(ff.axpy(alpha, gpu(a), gpu(b)).cpu().numpy(), oracle.axpy(alpha, a.numpy(), b.numpy()))
    dout = gpu(torch.from_numpy(alpha.copy()))
    dx, dy = ff.dot_backward(dout, gpu(a), gpu(b))
    wdx, wdy = oracle.dot_backward(alpha, a.numpy(), b.numpy())
    same_bits(dx.cpu().numpy(), wdx)
    same_bits(dy.cpu().numpy(), wdy)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 7, 257, 4099, 65537])
@pytest.mark.parametrize("offset", [0, 1])
def test_ragged_and_misaligned(cfg0, n, offset):
    """Lengths around the vector width and arrays starting 8 bytes past a
    16-byte boundary (one-element scalar head)."""
    a = gpu(cfg0.a[: n + 1])[offset:offset + n]
    b = gpu(cfg0.b[: n + 1])[offset:offset + n]
    an, bn = a.cpu().numpy(), b.cpu().numpy()
    same_bits(ff.add(a, b).cpu().numpy(), oracle.add22(an, bn))
    same_bits(ff.mul(a, b).cpu().numpy(), oracle.mul22(an, bn))
    same_bits(ff.div(a, b).cpu().numpy(), oracle.div22(an, bn))
    asq = gpu(cfg0.a_sqrt[: n + 1])[offset:offset + n]
    same_bits(ff.sqrt(asq).cpu().numpy(), oracle.sqrt22(asq.cpu().numpy()))


def test_mixed_alignment_scalar_path(cfg0):
    n = 10001
    a = gpu(cfg0.a[: n + 1])
    b = gpu(cfg0.b[: n + 1])
    out = torch.empty((n + 1, 2), dtype=torch.float32, device=DEV)
    # a aligned, b and out 8 bytes off: offsets modulo 16 differ
    ff.add(a[:n], b[1:], out=out[1:])
    same_bits(out[1:].cpu().numpy(), oracle.add22(cfg0.a[:n].numpy(), cfg0.b[1:n + 1].numpy()))


def test_in_place(cfg0):
    n = 12345
    a = gpu(cfg0.a[:n]).clone()
    b = gpu(cfg0.b[:n])
    want = oracle.mul22(cfg0.a[:n].numpy(), cfg0.b[:n].numpy())
    ff.mul(a, b, out=a)
    same_bits(a.cpu().numpy(), want)


def test_special_values():
    f = np.float32
    vals = [0.0, -0.0, 1.0, -1.0, 2.0 ** -149, -(2.0 ** -149), 2.0 ** -126, 3.0e-39, 1e38, -1e38,
            np.inf, -np.inf, np.nan, 2.0 ** 100, 2.0 ** -100, 1.5, 3.0]
    lo_vals = [0.0, -0.0, 2.0 ** -149, 1e-30, -1e-20]
    a = np.array([(h, l) for h in vals for l in lo_vals], f)
    A = np.repeat(a, len(a), axis=0)
    B = np.tile(a, (len(a), 1))
    for op, ref in (("add", oracle.add22), ("mul", oracle.mul22), ("div", oracle.div22)):
        got = getattr(ff, op)(gpu(torch.from_numpy(A)), gpu(torch.from_numpy(B))).cpu().numpy()
        same_bits(got, ref(A, B))
    same_bits(ff.sqrt(gpu(torch.from_numpy(a))).cpu().numpy(), oracle.sqrt22(a))
    ab = np.stack([A[:, 0], B[:, 0]], 1)
    same_bits(ff.add12(gpu(torch.from_numpy(ab))).cpu().numpy(), oracle.add12(ab))
    same_bits(ff.mul12(gpu(torch.from_numpy(ab))).cpu().numpy(), oracle.mul12(ab))


def test_add22_low_part_order_worked_examples():
    """The hand-derived cases in which the order of Add22's two low parts
    (Section 4.1, Add22 theorem) decides the bits: the GPU's select form
    gives the paper's order in both branches, like the oracle."""
    from test_oracle_pins import add22_low_part_order_cases
    a, b, want = add22_low_part_order_cases()
    got = ff.add(gpu(torch.from_numpy(a)), gpu(torch.from_numpy(b))).cpu().numpy()
    same_bits(got, want)
    same_bits(got, oracle.add22(a, b))


def test_subnormal_results_not_flushed():
    ab = np.array([[2.0 ** -140, 2.0 ** -149], [2.0 ** -70, 2.0 ** -70], [1e-20, 1e-20]], np.float32)
    got = ff.add12(gpu(torch.from_numpy(ab))).cpu().numpy()
    assert got[0, 0] != 0
    got = ff.mul12(gpu(torch.from_numpy(ab))).cpu().numpy()
    assert got[1, 0] == np.float32(2.0 ** -140)
    same_bits(got, oracle.mul12(ab))


# ---------------------------------------------------------------------------
# reductions
# ---------------------------------------------------------------------------

def shape_of(x, y):
    import ctypes
    g, h, v = ctypes.c_uint(), ctypes.c_int(), ctypes.c_int()
    _lib.call("ff_reduce_launch_shape", x.data_ptr(), None if y is None else y.data_ptr(), x.shape[0],
              ctypes.byref(g), ctypes.byref(h), ctypes.byref(v))
    return g.value, h.value, bool(v.value)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 1000, 4099, 300001])
@pytest.mark.parametrize("offset", [0, 1])
def test_dot_and_sum_replay_bitexact(cfg0, n, offset):
    x = gpu(cfg0.a[: n + 1])[offset:offset + n]
    y = gpu(cfg0.b[: n + 1])[offset:offset + n]
    xn, yn = x.cpu().numpy(), y.cpu().numpy()
    import replay
    g, h, v = shape_of(x, y)
    same_bits(ff.dot(x, y).cpu().numpy(), replay.reduce_replay(oracle.mul22(xn, yn), g, h, v))
    g, h, v = shape_of(x, None)
    same_bits(ff.sum(x).cpu().numpy(), replay.reduce_replay(xn, g, h, v))


def test_dot_and_sum_full_size_replay_bitexact():
    """At the benchmark's size (2^26 values, cond 1e12), ff_dot and ff_sum
    match the replay of their documented order bit for bit."""
    import replay
    n = 1 << 26
    g_ = inputs.ill_dot(n, 1e12, inputs.seed_for(2, 12), device=DEV)
    xn, yn = g_.x.cpu().numpy(), g_.y.cpu().numpy()
    terms = _oracle_threaded(oracle.mul22, xn, yn)
    g, h, v = shape_of(g_.x, g_.y)
    same_bits(ff.dot(g_.x, g_.y).cpu().numpy(), replay.reduce_replay(terms, g, h, v))
    g, h, v = shape_of(g_.x, None)
    same_bits(ff.sum(g_.x).cpu().numpy(), replay.reduce_replay(xn, g, h, v))
    del g_, terms
    torch.cuda.empty_cache()


@pytest.mark.parametrize("offset", [0, 1])
def test_reductions_with_specials_follow_the_replay(cfg0, offset):
    """Infinities, NaN, values whose products overflow, subnormals and signed
    zeros planted at the head, in the middle and at the tail: ff_dot and
    ff_sum give the bits of the replay of their order (NaN as NaN)."""
    import replay
    n = 70001
    x = cfg0.a[: n + 1].clone()
    y = cfg0.b[: n + 1].clone()
    plants = {0: (float("inf"), 0.0), 1: (-0.0, -0.0), 3: (1e-40, 0.0), 4097: (3e38, 1e31),
              35000: (float("nan"), 0.0), 35001: (-float("inf"), 0.0), n - 1: (2.0 ** -149, 0.0), n: (-3e38, 0.0)}
    for i, v in plants.items():
        x[i] = torch.tensor(v)
        y[i] = torch.tensor((v[0] if i % 2 else 1.5, 0.0))
    for lo in (0, 1):                       # with and without the NaN
        xs = gpu(x)[offset:offset + n]
        ys = gpu(y)[offset:offset + n]
        if lo:
            xs = xs.clone(); xs[35000 - offset] = torch.tensor((2.0, 0.0))
        xn, yn = xs.cpu().numpy(), ys.cpu().numpy()
        g, h, v = shape_of(xs, ys)
        same_bits(ff.dot(xs, ys).cpu().numpy(), replay.reduce_replay(oracle.mul22(xn, yn), g, h, v))
        g, h, v = shape_of(xs, None)
        same_bits(ff.sum(xs).cpu().numpy(), replay.reduce_replay(xn, g, h, v))


def test_dot_mixed_alignment_replay(cfg0):
    n = 70001
    x = gpu(cfg0.a[: n + 1])[:n]
    y = gpu(cfg0.b[: n + 1])[1:]
    import replay
    g, h, v = shape_of(x, y)
    assert not v
    want = replay.reduce_replay(oracle.mul22(x.cpu().numpy(), y.cpu().numpy()), g, h, v)
    same_bits(ff.dot(x, y).cpu().numpy(), want)


@pytest.mark.parametrize("cond", [1e3, 1e6, 1e9, 1e12])
def test_dot_ill_conditioned_within_bound(cond):
    n = 1 << 22
    g = inputs.ill_dot(n, cond, inputs.seed_for(2, int(np.log10(cond))))
    x, y = gpu(g.x), gpu(g.y)
    r = ff.dot(x, y).cpu().numpy()
    s_hi, s_lo, A, E = oracle.exact_dot(g.x.numpy(), g.y.numpy(), r)
    assert abs(E) <= n * 2.0 ** -46 * A
    # tree order: far inside the bound in practice
    assert abs(E) <= 64 * 2.0 ** -46 * A
    # deterministic
    same_bits(ff.dot(x, y).cpu().numpy(), r)


def test_sum_of_ones_and_n0():
    for n in (0, 1, 3, 1000, 1 << 20):
        x = torch.zeros((n, 2), dtype=torch.float32, device=DEV)
        x[:, 0] = 1.0
        r = ff.sum(x).cpu().numpy()
        assert r[0] == n and r[1] == 0


def test_autograd_dot():
    e = inputs.elementwise(50001, inputs.seed_for(2, 9))
    x = gpu(e.a).requires_grad_(True)
    y = gpu(e.b).requires_grad_(True)
    d = ff.ffdot(x, y)
    dout = inputs.scalar_ff(5)
    d.backward(gpu(dout))
    wdx, wdy = oracle.dot_backward(dout.numpy(), e.a.numpy(), e.b.numpy())
    same_bits(x.grad.cpu().numpy(), wdx)
    same_bits(y.grad.cpu().numpy(), wdy)


# ---------------------------------------------------------------------------
# GEMV
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m,n,k", [(37, 129, 1), (64, 256, 3), (200, 1000, 17), (33, 66, 64), (8, 7, 2)])
def test_gemv_within_bound(m, n, k):
    gi = inputs.gemv(m, n, k, inputs.seed_for(4, m + n + k))
    A, X, dY = gpu(gi.A), gpu(gi.X), gpu(gi.dY)
    Y = ff.gemv(A, X).cpu().numpy()
    An, Xn, dYn = gi.A.numpy(), gi.X.numpy(), gi.dY.numpy()
    for c in range(k):
        for r in range(0, m, max(1, m // 16)):
            _, _, Aabs, E = oracle.exact_dot(An[r], Xn[c], Y[c, r])
            assert abs(E) <= 64 * 2.0 ** -46 * Aabs + 1e-300
    dX = ff.gemv_t(A, dY).cpu().numpy()
    At = np.ascontiguousarray(An.transpose(1, 0, 2))
    for c in range(k):
        for j in range(0, n, max(1, n // 16)):
            _, _, Aabs, E = oracle.exact_dot(At[j], dYn[c], dX[c, j])
            assert abs(E) <= 64 * 2.0 ** -46 * Aabs + 1e-300


def test_gemv_autograd():
    gi = inputs.gemv(64, 96, 4, inputs.seed_for(4, 77))
    A = gpu(gi.A)
    X = gpu(gi.X).requires_grad_(True)
    Y = ff.ffgemv(A, X)
    dY = gpu(gi.dY)
    Y.backward(dY)
    want = ff.gemv_t(A, dY)
    same_bits(X.grad.cpu().numpy(), want.cpu().numpy())


# ---------------------------------------------------------------------------
# native baselines
# ---------------------------------------------------------------------------

def test_f64_and_f32_baselines(cfg0):
    a64 = inputs.ff_to_f64(cfg0.a).to(DEV)
    b64 = inputs.ff_to_f64(cfg0.b).to(DEV)
    assert torch.equal(ff.f64_add(a64, b64), a64 + b64)
    assert torch.equal(ff.f64_mul(a64, b64), a64 * b64)
    assert torch.equal(ff.f64_div(a64, b64), a64 / b64)
    s = a64.abs()
    assert torch.equal(ff.f64_sqrt(s), torch.sqrt(s))
    d = ff.f64_dot(a64, b64).item()
    ex = oracle.exact_dot(cfg0.a.numpy(), cfg0.b.numpy())
    assert abs(d - ex[0]) <= a64.numel() * 2.0 ** -53 * ex[2]
    a32 = gpu(cfg0.a[:, 0].contiguous())
    b32 = gpu(cfg0.b[:, 0].contiguous())
    c32 = gpu(cfg0.ab[:, 1].contiguous())
    same_bits(ff.f32_add(a32, b32).cpu().numpy(), oracle.fp32_add(a32.cpu().numpy(), b32.cpu().numpy()))
    same_bits(ff.f32_mul(a32, b32).cpu().numpy(), oracle.fp32_mul(a32.cpu().numpy(), b32.cpu().numpy()))
    same_bits(ff.f32_mad(a32, b32, c32).cpu().numpy(),
              oracle.fp32_mad(a32.cpu().numpy(), b32.cpu().numpy(), c32.cpu().numpy()))
    gi = inputs.gemv(40, 100, 3, 5)
    A64 = inputs.ff_to_f64(gi.A).to(DEV)
    X64 = inputs.ff_to_f64(gi.X).to(DEV)
    Y = ff.f64_gemv(A64, X64)
    torch.testing.assert_close(Y, X64 @ A64.T, rtol=1e-13, atol=0)


def test_gemv_and_f64_gemv_normwise_2m44():
    """The float-float GEMV and the binary64 baseline GEMV at the benchmark's
    row width (32768): every element within 2^-44 sum_j |A_rj x_j| of the
    exact value (superaccumulator), the per-row normwise reading of a
    relative error <= 2^-44."""
    m, n, k = 48, 32768, 4
    gi = inputs.gemv(m, n, k, inputs.seed_for(4, 150))
    A, X = gi.A.numpy(), gi.X.numpy()
    Y = ff.gemv(gpu(gi.A), gpu(gi.X)).cpu().numpy()
    Y64 = ff.f64_gemv(inputs.ff_to_f64(gi.A).to(DEV), inputs.ff_to_f64(gi.X).to(DEV)).cpu().numpy()
    worst = worst64 = 0.0
    for c in range(k):
        for r in range(m):
            s_hi, s_lo, Aabs, E = oracle.exact_dot(A[r], X[c], Y[c, r])
            worst = max(worst, abs(E) / Aabs)
            e64 = abs((Y64[c, r] - s_hi) - s_lo)   # binary128 exact value as a double pair
            worst64 = max(worst64, e64 / Aabs)
    assert worst <= 2.0 ** -44 and worst64 <= 2.0 ** -44, (worst, worst64)


# ---------------------------------------------------------------------------
# full size (2^28 values), sampled against the oracle
# ---------------------------------------------------------------------------

def test_full_size_sampled_bitexact():
    n = 1 << 28
    e = inputs.elementwise(n, inputs.seed_for(1, 0), device=DEV)
    g = torch.Generator().manual_seed(1234)
    idx = torch.cat([torch.arange(4096), torch.randint(0, n, (1 << 20,), generator=g),
                     torch.arange(n - 4096, n)]).to(DEV)
    take = lambda t: t[idx].cpu().numpy()
    a, b, ab, asq = take(e.a), take(e.b), take(e.ab), take(e.a_sqrt)
    out = torch.empty_like(e.a)
    same_bits(take(ff.add12(e.ab, out=out)), oracle.add12(ab))
    same_bits(take(ff.mul12(e.ab, out=out)), oracle.mul12(ab))
    same_bits(take(ff.add(e.a, e.b, out=out)), oracle.add22(a, b))
    same_bits(take(ff.mul(e.a, e.b, out=out)), oracle.mul22(a, b))
    same_bits(take(ff.div(e.a, e.b, out=out)), oracle.div22(a, b))
    same_bits(take(ff.sqrt(e.a_sqrt, out=out)), oracle.sqrt22(asq))
    # divisor floor of the operators holds for the generated divisors
    assert e.b[:, 0].abs().min().item() >= 2.0 ** -60
    del out, e
    torch.cuda.empty_cache()


def test_mul12_mul22_match_dekker_split_form(cfg0):
    """The GPU's fused Mul12 against the paper's Split-based (Dekker) form of
    the oracle: the same pair (RN(ab), ab - RN(ab)) wherever neither part
    under- or overflows (|a|, |b| in [2^-60, 2^60], |ab| >= 2^-100), up to
    the sign of a zero error term; likewise Mul22 built on either form."""
    import test_oracle_pins as pins
    S = pins.subset_floats()
    ab = np.concatenate([pins.all_pairs(S), cfg0.ab.numpy()])
    p = ab[:, 0].astype(np.float64) * ab[:, 1].astype(np.float64)
    dom = np.all((np.abs(ab) >= 2.0 ** -60) & (np.abs(ab) <= 2.0 ** 60), axis=1) & (np.abs(p) >= 2.0 ** -100)
    ab = np.ascontiguousarray(ab[dom])
    pins.assert_same_up_to_zero_sign(ff.mul12(gpu(torch.from_numpy(ab))).cpu().numpy(), oracle.mul12_dekker(ab))
    a, b = cfg0.a.numpy(), cfg0.b.numpy()
    pins.assert_same_up_to_zero_sign(ff.mul(gpu(cfg0.a), gpu(cfg0.b)).cpu().numpy(), oracle.mul22_dekker(a, b))


def test_bruteforce_subsets_bitexact():
    """Every ordered pair of the oracle pins' brute-force subsets (extreme
    significands 0x800000..0x80000F and 0xFFFFF0..0xFFFFFF, exponents -30..30,
    both signs; float-float values with low parts 0, about ulp/2 and 2^-30
    hi), bit for bit on the GPU."""
    import test_oracle_pins as pins
    S = pins.subset_floats()
    ab = pins.all_pairs(S)
    abd = gpu(torch.from_numpy(ab))
    same_bits(ff.add12(abd).cpu().numpy(), oracle.add12(ab))
    same_bits(ff.mul12(abd).cpu().numpy(), oracle.mul12(ab))
    F = pins.ff_subset()
    i, j = np.meshgrid(np.arange(F.shape[0]), np.arange(F.shape[0]), indexing="ij")
    a, b = np.ascontiguousarray(F[i.ravel()]), np.ascontiguousarray(F[j.ravel()])
    ad, bd = gpu(torch.from_numpy(a)), gpu(torch.from_numpy(b))
    same_bits(ff.add(ad, bd).cpu().numpy(), oracle.add22(a, b))
    same_bits(ff.mul(ad, bd).cpu().numpy(), oracle.mul22(a, b))
    same_bits(ff.div(ad, bd).cpu().numpy(), oracle.div22(a, b))
    same_bits(ff.add_accurate(ad, bd).cpu().numpy(), oracle.add22_accurate(a, b))
    s = F.copy()
    s[s[:, 0] < 0] *= -1
    same_bits(ff.sqrt(gpu(torch.from_numpy(s))).cpu().numpy(), oracle.sqrt22(s))


def _oracle_threaded(fn, *arrays, threads=None):
    """The oracle function over contiguous chunks on all host cores (its C
    loops release the GIL); the result equals one call on the whole arrays."""
    import concurrent.futures as cf
    import os
    threads = threads or max(1, len(os.sched_getaffinity(0)))
    n = arrays[0].shape[0]
    cuts = [n * i // threads for i in range(threads + 1)]
    with cf.ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda i: fn(*(a[cuts[i]:cuts[i + 1]] for a in arrays)), range(threads)))
    return np.concatenate(parts)


def test_full_size_every_value_bitexact():
    """All 2^28 results of each of the six operators at the benchmark's size,
    bit for bit against the oracle (in chunks of 2^26 values)."""
    n = 1 << 28
    e = inputs.elementwise(n, inputs.seed_for(1, 0), device=DEV)
    out = torch.empty_like(e.a)
    cases = [("add12", lambda: ff.add12(e.ab, out=out), oracle.add12, ("ab",)),
             ("mul12", lambda: ff.mul12(e.ab, out=out), oracle.mul12, ("ab",)),
             ("add", lambda: ff.add(e.a, e.b, out=out), oracle.add22, ("a", "b")),
             ("mul", lambda: ff.mul(e.a, e.b, out=out), oracle.mul22, ("a", "b")),
             ("div", lambda: ff.div(e.a, e.b, out=out), oracle.div22, ("a", "b")),
             ("sqrt", lambda: ff.sqrt(e.a_sqrt, out=out), oracle.sqrt22, ("a_sqrt",))]
    chunk = 1 << 26
    for name, gpu_op, orc_op, keys in cases:
        gpu_op()
        torch.cuda.synchronize()
        for lo in range(0, n, chunk):
            ins = [getattr(e, k)[lo:lo + chunk].cpu().numpy() for k in keys]
            same_bits(out[lo:lo + chunk].cpu().numpy(), _oracle_threaded(orc_op, *ins))
    del out, e
    torch.cuda.empty_cache()


@pytest.mark.parametrize("m,n,k", [(37, 1000, 3), (20, 999, 2), (5, 64, 17), (1, 1, 1), (9, 33, 1), (301, 1000, 2),
                                   (64, 130, 7), (33, 2, 5), (17, 66, 1)])
def test_gemv_bitexact_vs_order_replay(m, n, k):
    """ff_gemv bit for bit against the replay of its documented warp order."""
    import replay
    gi = inputs.gemv(m, n, k, inputs.seed_for(4, 120 + n % 7))
    Y = ff.gemv(gpu(gi.A), gpu(gi.X)).cpu().numpy()
    same_bits(Y, replay.gemv_warp_replay(gi.A.numpy(), gi.X.numpy(), vec=(n % 2 == 0)))


@pytest.mark.parametrize("m,n,k", [(4096, 256, 3), (3000, 130, 2), (70, 513, 5), (31, 8, 1), (5000, 770, 7),
                                   (4099, 66, 4), (1027, 1030, 6), (2500, 518, 9), (8191, 64, 1)])
def test_gemv_t_bitexact_vs_order_replay(m, n, k):
    """ff_gemv_t bit for bit against the replay of its row-block order (the
    row-block count read from ff_gemv_t_launch_shape)."""
    import ctypes
    import replay
    gi = inputs.gemv(m, n, k, inputs.seed_for(4, 130 + k))
    A, dY = gpu(gi.A), gpu(gi.dY)
    nrb, vec = ctypes.c_int64(), ctypes.c_int()
    _lib.call("ff_gemv_t_launch_shape", A.data_ptr(), m, n, n, k, ctypes.byref(nrb), ctypes.byref(vec))
    assert nrb.value >= 1 and bool(vec.value) == (n % 2 == 0)
    dX = ff.gemv_t(A, dY).cpu().numpy()
    same_bits(dX, replay.gemv_t_replay(gi.A.numpy(), gi.dY.numpy(), nrb.value))
    if m >= 4096:
        assert nrb.value > 1  # the multi-block combine is exercised


@pytest.mark.parametrize("n", [1000, 999])
def test_gemv_result_does_not_depend_on_k(n):
    """Every right-hand side is reduced in the same order whatever k and the
    tile widths are: k = 20 in one call (tiles 8 + 8 + 4) equals 20 one-column
    calls bit for bit, with 16-byte access (n even) and without (n odd)."""
    gi = inputs.gemv(300, n, 20, inputs.seed_for(4, 95 + n % 2))
    A, X = gpu(gi.A), gpu(gi.X)
    Y = ff.gemv(A, X).cpu().numpy()
    for c in range(20):
        same_bits(Y[c], ff.gemv(A, X[c:c + 1].contiguous())[0].cpu().numpy())


@pytest.mark.parametrize("m,n,k", [(33, 64, 1), (17, 129, 5), (64, 256, 64), (17, 129, 3), (301, 1000, 4),
                                   (300, 998, 2), (257, 66, 7), (256, 514, 8), (1000, 2050, 5), (999, 130, 6),
                                   (40, 20, 9), (301, 130, 12), (256, 66, 16), (33, 64, 15), (17, 129, 12),
                                   (70, 50, 17), (100, 130, 13), (99, 64, 10), (129, 66, 11), (5, 2, 3),
                                   (1, 4, 12), (2, 2, 1), (66, 64, 21), (35, 130, 19), (41, 32, 20),
                                   (7, 2, 13), (130, 66, 22), (33, 65, 19), (5001, 4, 17), (3, 5000, 20)])
def test_gemv_dA_bitexact(m, n, k):
    gi = inputs.gemv(m, n, k, inputs.seed_for(4, 50 + k))
    dA = ff.gemv_dA(gpu(gi.dY), gpu(gi.X)).cpu().numpy()
    same_bits(dA, oracle.gemv_dA(gi.dY.numpy(), gi.X.numpy()))


@pytest.mark.parametrize("m,n,k", [(130, 66, 1), (129, 128, 2), (64, 70, 3), (66, 64, 8), (65, 66, 12),
                                   (65, 66, 20)])
def test_gemv_dA_special_values_bitexact(m, n, k):
    """dA's first term takes a shortcut for finite normalised products and
    the full Add22 from (0, 0) otherwise: signed zeros, subnormals,
    overflowing products, infinities and NaN planted in dY and X give the
    oracle's bits (NaN == NaN), for warps that see them and warps that do
    not."""
    gi = inputs.gemv(m, n, k, inputs.seed_for(4, 70 + k))
    dY, X = gi.dY.numpy().copy(), gi.X.numpy().copy()
    rng = np.random.default_rng(17 + k)
    specials = np.array([(0.0, 0.0), (-0.0, 0.0), (-0.0, -0.0), (2.0 ** -149, 0.0), (-(2.0 ** -140), 2.0 ** -149),
                         (3e38, 1e30), (-3e38, 0.0), (np.inf, 0.0), (-np.inf, 0.0), (np.nan, 0.0), (1.0, np.nan),
                         (2.0 ** 100, 2.0 ** 76), (1.0, 1.0)], np.float32)
    for arr, rows in ((dY, m), (X, n)):
        for _ in range(max(4, rows // 8)):
            c, i = rng.integers(0, k), rng.integers(0, rows)
            arr[c, i] = specials[rng.integers(0, len(specials))]
    dA = ff.gemv_dA(gpu(torch.from_numpy(dY)), gpu(torch.from_numpy(X))).cpu().numpy()
    same_bits(dA, oracle.gemv_dA(dY, X))


def test_gemv_family_empty_sums_and_empty_outputs():
    """Degenerate sizes: with n = 0 every element of Y = A X is an empty sum,
    (+0, +0), and so is every element of dX = A^T dY with m = 0; outputs
    with no elements (m = 0 for Y and dA, n = 0 for dA) are returned empty
    and nothing is written."""
    Y = torch.full((3, 5, 2), 7.25, device=DEV)
    ff.gemv(torch.empty((5, 0, 2), device=DEV), torch.empty((3, 0, 2), device=DEV), out=Y)
    dX = torch.full((3, 6, 2), 7.25, device=DEV)
    ff.gemv_t(torch.empty((0, 6, 2), device=DEV), torch.empty((3, 0, 2), device=DEV), out=dX)
    torch.cuda.synchronize()
    assert torch.count_nonzero(Y.view(torch.int32)) == 0
    assert torch.count_nonzero(dX.view(torch.int32)) == 0
    gi = inputs.gemv(5, 6, 3, inputs.seed_for(4, 170))
    A, X, dY = gpu(gi.A), gpu(gi.X), gpu(gi.dY)
    assert ff.gemv(A[:0].contiguous(), X).shape == (3, 0, 2)
    assert ff.gemv_t(A[:, :0].contiguous(), dY).shape == (3, 0, 2)
    assert ff.gemv_dA(dY[:, :0].contiguous(), X).shape == (0, 6, 2)
    assert ff.gemv_dA(dY, X[:, :0].contiguous()).shape == (5, 0, 2)
    torch.cuda.synchronize()


def test_gemv_autograd_weight_gradient():
    gi = inputs.gemv(48, 80, 3, inputs.seed_for(4, 60))
    A = gpu(gi.A).requires_grad_(True)
    X = gpu(gi.X).requires_grad_(True)
    Y = ff.ffgemv(A, X)
    Y.backward(gpu(gi.dY))
    same_bits(A.grad.cpu().numpy(), oracle.gemv_dA(gi.dY.numpy(), gi.X.numpy()))
    same_bits(X.grad.cpu().numpy(), ff.gemv_t(gpu(gi.A), gpu(gi.dY)).cpu().numpy())


# ---------------------------------------------------------------------------
# maximum sizes: more than 2^32 values (64-bit indexing end to end)
# ---------------------------------------------------------------------------

def _big_pattern(n, scale, dev):
    """Cheap deterministic float-float values for very large n: hi = 1 + (i
    mod 4093) 2^-12 times `scale`, lo = hi 2^-30 (i mod 7 - 3) / 4 (exact)."""
    i = torch.arange(n, device=dev, dtype=torch.int64)
    hi = (1.0 + (i % 4093).to(torch.float32) * 2.0 ** -12) * scale
    lo = hi * ((i % 7 - 3).to(torch.float32) * 2.0 ** -32)
    del i
    return torch.stack([hi, lo], dim=1)


def test_more_than_2_32_values_elementwise_and_dot():
    free, _ = torch.cuda.mem_get_info()
    n = (1 << 32) + 5
    if free < (180 << 30):
        pytest.skip("needs ~180 GB of free device memory (three 32 GiB arrays and temporaries)")
    a = _big_pattern(n, 1.0, DEV)
    b = _big_pattern(n, -0.75, DEV)
    out = ff.add(a, b)
    idx = torch.cat([torch.arange(8), torch.randint(0, n, (1 << 16,), generator=torch.Generator().manual_seed(5)),
                     torch.arange((1 << 32) - 4, n)]).to(DEV)
    an, bn = a[idx].cpu().numpy(), b[idx].cpu().numpy()
    same_bits(out[idx].cpu().numpy(), oracle.add22(an, bn))
    ff.mul(a, b, out=out)
    same_bits(out[idx].cpu().numpy(), oracle.mul22(an, bn))
    del out, b
    torch.cuda.empty_cache()
    # sum of n ones: every partial sum is an integer below 2^48, exact in
    # float-float, so the result is exactly (RN32(n), n - RN32(n))
    a.zero_()
    a[:, 0] = 1.0
    r = ff.sum(a).cpu().numpy()
    hi = np.float32(n)
    assert r[0] == hi and float(r[1]) == float(n - float(hi))
    r = ff.dot(a, a).cpu().numpy()
    assert r[0] == hi and float(r[1]) == float(n - float(hi))
    del a
    torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# guard regions: no kernel writes outside its output
# ---------------------------------------------------------------------------
GUARD = 64
SENTINEL = np.array([0x7FC0DEAD], dtype=np.uint32).view(np.float32)[0]


def guarded(rows, offset=0, width=2):
    """A view of `rows` float32 rows inside a buffer with GUARD sentinel rows
    on both sides (the view starts `offset` rows past the guard)."""
    buf = torch.full((rows + 2 * GUARD + offset, width), float(SENTINEL), dtype=torch.float32, device=DEV)
    view = buf[GUARD + offset:GUARD + offset + rows]
    return buf, view


def guards_intact(buf, rows, offset=0):
    b = buf.cpu().numpy().view(np.uint32)
    s = np.array([0x7FC0DEAD], np.uint32)[0]
    return bool((b[:GUARD + offset] == s).all() and (b[GUARD + offset + rows:] == s).all())


@pytest.mark.parametrize("n", [1, 2, 3, 5, 4099, 65537])
@pytest.mark.parametrize("offset", [0, 1])
def test_outputs_stay_inside_their_bounds(cfg0, n, offset):
    a = gpu(cfg0.a[:n])
    b = gpu(cfg0.b[:n])
    for name, fn in (("add", lambda o: ff.add(a, b, out=o)), ("mul", lambda o: ff.mul(a, b, out=o)),
                     ("div", lambda o: ff.div(a, b, out=o)), ("sqrt", lambda o: ff.sqrt(a.abs(), out=o)),
                     ("add_accurate", lambda o: ff.add_accurate(a, b, out=o)),
                     ("add12", lambda o: ff.add12(gpu(cfg0.ab[:n]), out=o)),
                     ("mul12", lambda o: ff.mul12(gpu(cfg0.ab[:n]), out=o)),
                     ("axpy", lambda o: ff.axpy((1.5, 0.0), a, b, out=o))):
        buf, view = guarded(n, offset)
        fn(view)
        torch.cuda.synchronize()
        assert guards_intact(buf, n, offset), name
    bx, dx = guarded(n, offset)
    by, dy = guarded(n, offset)
    ff.dot_backward(gpu(torch.tensor([1.25, 0.0])), a, b, dx, dy)
    torch.cuda.synchronize()
    assert guards_intact(bx, n, offset) and guards_intact(by, n, offset)
    br, r = guarded(1, offset)
    ff.dot(a, b, out=r.reshape(2))
    ff.sum(a, out=r.reshape(2))
    torch.cuda.synchronize()
    assert guards_intact(br, 1, offset)


@pytest.mark.parametrize("m,n,k", [(9, 7, 1), (33, 130, 5), (70, 64, 17)])
def test_gemv_outputs_stay_inside_their_bounds(m, n, k):
    gi = inputs.gemv(m, n, k, inputs.seed_for(4, 90 + k))
    A, X, dY = gpu(gi.A), gpu(gi.X), gpu(gi.dY)
    buf, view = guarded(k * m)
    ff.gemv(A, X, out=view.view(k, m, 2))
    torch.cuda.synchronize()
    assert guards_intact(buf, k * m)
    buf, view = guarded(k * n)
    ff.gemv_t(A, dY, out=view.view(k, n, 2))
    torch.cuda.synchronize()
    assert guards_intact(buf, k * n)
    buf, view = guarded(m * n)
    ff.gemv_dA(dY, X, out=view.view(m, n, 2))
    torch.cuda.synchronize()
    assert guards_intact(buf, m * n)


# ---------------------------------------------------------------------------
# GEMV family with leading dimensions larger than the sizes (through the C ABI)
# ---------------------------------------------------------------------------

def _padded(rows, cols, ld, src=None, fill=-7.25):
    """A (rows, ld, 2) device buffer whose first `cols` columns hold `src`
    (or stay `fill`) and whose padding columns hold `fill`."""
    buf = torch.full((rows, ld, 2), fill, dtype=torch.float32, device=DEV)
    if src is not None:
        buf[:, :cols] = src.to(DEV)
    return buf


@pytest.mark.parametrize("m,n,k,pad", [(300, 258, 3, 2), (301, 130, 9, 4), (257, 66, 16, 2), (129, 98, 2, 1)])
def test_gemv_family_with_leading_dimensions(m, n, k, pad):
    """ff_gemv, ff_gemv_t and ff_gemv_dA on operands stored with row strides
    (lda, ldx, lddy, ldy, lddx, ldda) `pad` values wider than the sizes: with
    an even pad every kernel takes the same path as for packed operands and
    gives the same bits; with an odd pad the 8-byte paths run, checked
    against the replays of their order (ff_gemv, ff_gemv_t) and the oracle
    (ff_gemv_dA, elementwise).  No padding value is touched."""
    import ctypes
    import replay
    gi = inputs.gemv(m, n, k, inputs.seed_for(4, 150 + pad))
    stream = torch.cuda.current_stream().cuda_stream
    A = _padded(m, n, n + pad, gi.A)
    X = _padded(k, n, n + pad, gi.X)
    dY = _padded(k, m, m + pad, gi.dY)
    Y = _padded(k, m, m + pad)
    dX = _padded(k, n, n + pad)
    dA = _padded(m, n, n + pad)
    _lib.call("ff_gemv", A.data_ptr(), m, n, n + pad, X.data_ptr(), n + pad, k, Y.data_ptr(), m + pad, stream)
    wsb = _lib.load().ff_gemv_t_workspace_bytes(m, n, k)
    ws = torch.zeros(max(wsb, 256), dtype=torch.uint8, device=DEV)
    _lib.call("ff_gemv_t", A.data_ptr(), m, n, n + pad, dY.data_ptr(), m + pad, k, dX.data_ptr(), n + pad,
              ws.data_ptr(), ws.numel(), stream)
    _lib.call("ff_gemv_dA", dY.data_ptr(), m, m + pad, X.data_ptr(), n, n + pad, k, dA.data_ptr(), n + pad, stream)
    torch.cuda.synchronize()
    for buf, cols in ((Y, m), (dX, n), (dA, n)):
        tail = buf[:, cols:].cpu().numpy()
        assert np.all(tail == np.float32(-7.25)), "padding overwritten"
    Yg, dXg, dAg = Y[:, :m].cpu().numpy(), dX[:, :n].cpu().numpy(), dA[:, :n].cpu().numpy()
    if pad % 2 == 0:
        Ad, Xd, dYd = gpu(gi.A), gpu(gi.X), gpu(gi.dY)
        same_bits(Yg, ff.gemv(Ad, Xd).cpu().numpy())
        same_bits(dXg, ff.gemv_t(Ad, dYd).cpu().numpy())
        same_bits(dAg, ff.gemv_dA(dYd, Xd).cpu().numpy())
    else:
        same_bits(Yg, replay.gemv_warp_replay(gi.A.numpy(), gi.X.numpy(), vec=False))
        nrb, vec = ctypes.c_int64(), ctypes.c_int()
        _lib.call("ff_gemv_t_launch_shape", A.data_ptr(), m, n, n + pad, k, ctypes.byref(nrb), ctypes.byref(vec))
        assert vec.value == 0
        same_bits(dXg, replay.gemv_t_replay(gi.A.numpy(), gi.dY.numpy(), nrb.value))
        same_bits(dAg, oracle.gemv_dA(gi.dY.numpy(), gi.X.numpy()))
