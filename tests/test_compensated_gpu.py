"""Parity of the rows beyond the paper's operator set: the accurate
float-float addition (bit-exact against the oracle) and the compensated
Sum2 / Dot2 of binary32 vectors (bit-exact against a replay of the
documented order, within the error bound of the exact value)."""
import ctypes
import math

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
    eq = (got.view(np.uint32) == want.view(np.uint32)) | nan
    assert eq.all(), f"{(~eq).sum()} mismatches"


@pytest.mark.parametrize("n", [0, 1, 3, 4099, 1 << 20])
@pytest.mark.parametrize("offset", [0, 1])
def test_add_accurate_bitexact(n, offset):
    import paper_cs_0603115_gb300 as ff
    e = inputs.elementwise(n + 1, inputs.seed_for(0, 30), cancel_frac=0.3)
    a = e.a.to(DEV)[offset:offset + n]
    b = e.b.to(DEV)[offset:offset + n]
    same_bits(ff.add_accurate(a, b).cpu().numpy(), oracle.add22_accurate(a.cpu().numpy(), b.cpu().numpy()))


def test_add_accurate_specials():
    import paper_cs_0603115_gb300 as ff
    vals = [0.0, -0.0, 1.0, -1.0, 2.0 ** -149, 1e38, -1e38, np.inf, -np.inf, np.nan, 3.0, 2.0 ** -100]
    lo = [0.0, 2.0 ** -149, -1e-20]
    a = np.array([(h, l) for h in vals for l in lo], np.float32)
    A = np.repeat(a, len(a), axis=0)
    B = np.tile(a, (len(a), 1))
    got = ff.add_accurate(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)).cpu().numpy()
    same_bits(got, oracle.add22_accurate(A, B))


def _shape(x, y):
    from paper_cs_0603115_gb300 import _lib
    g, h, v = ctypes.c_uint(), ctypes.c_int(), ctypes.c_int()
    _lib.call("ff_reduce2_launch_shape", x.data_ptr(), None if y is None else y.data_ptr(), x.numel(),
              ctypes.byref(g), ctypes.byref(h), ctypes.byref(v))
    return g.value, h.value, bool(v.value)


@pytest.mark.parametrize("n", [0, 1, 5, 1001, 70003, 1 << 20])
@pytest.mark.parametrize("offset", [0, 1, 3])
def test_dot2_sum2_replay_bitexact(n, offset):
    import paper_cs_0603115_gb300 as ff
    import replay
    g = inputs.ill_dot_f32(max(n, 4) + 3, 1e9, inputs.seed_for(5, 50 + n % 7))
    x = g.x.to(DEV)[offset:offset + n]
    y = g.y.to(DEV)[offset:offset + n]
    xn, yn = x.cpu().numpy(), y.cpu().numpy()
    pol = replay.Dot2Policy()
    gr, h, v = _shape(x, y)
    terms = oracle.mul12(np.stack([xn, yn], 1)) if n else np.zeros((0, 2), np.float32)
    same_bits(ff.dot2(x, y).cpu().numpy(), replay.reduce_replay(terms, gr, h, v, pol))
    gr, h, v = _shape(x, None)
    terms = np.stack([xn, np.zeros_like(xn)], 1)
    same_bits(ff.sum2(x).cpu().numpy(), replay.reduce_replay(terms, gr, h, v, pol))


def test_dot2_sum2_full_size_replay_bitexact():
    """The benchmark's size: 2^26 binary32 values at cond 1e12."""
    import paper_cs_0603115_gb300 as ff
    import replay
    n = 1 << 26
    g = inputs.ill_dot_f32(n, 1e12, inputs.seed_for(5, 12), device=DEV)
    xn, yn = g.x.cpu().numpy(), g.y.cpu().numpy()
    pol = replay.Dot2Policy()
    gr, h, v = _shape(g.x, g.y)
    same_bits(ff.dot2(g.x, g.y).cpu().numpy(), replay.reduce_replay(oracle.mul12(np.stack([xn, yn], 1)), gr, h, v, pol))
    gr, h, v = _shape(g.x, None)
    same_bits(ff.sum2(g.x).cpu().numpy(), replay.reduce_replay(np.stack([xn, np.zeros_like(xn)], 1), gr, h, v, pol))


def test_dot2_sum2_with_specials_follow_the_replay():
    """Sum2 / Dot2 on binary32 vectors holding infinities, NaN, overflowing
    products, subnormals and signed zeros: the bits of the replay."""
    import paper_cs_0603115_gb300 as ff
    import replay
    n = 100003
    g = inputs.ill_dot_f32(n, 1e6, inputs.seed_for(5, 77))
    x, y = g.x.clone(), g.y.clone()
    for i, v in {0: float("inf"), 2: -0.0, 5: 1e-42, 999: 3e38, 50000: float("nan"), 50001: -float("inf"),
                 n - 2: 2.0 ** -149, n - 1: -3e38}.items():
        x[i] = v
        y[i] = v if i % 3 else 2.0
    for drop_nan in (False, True):
        if drop_nan:
            x[50000] = 1.0
        xd, yd = x.to(DEV), y.to(DEV)
        pol = replay.Dot2Policy()
        gr, h, v = _shape(xd, yd)
        want = replay.reduce_replay(oracle.mul12(np.stack([x.numpy(), y.numpy()], 1)), gr, h, v, pol)
        same_bits(ff.dot2(xd, yd).cpu().numpy(), want)
        gr, h, v = _shape(xd, None)
        want = replay.reduce_replay(np.stack([x.numpy(), np.zeros(n, np.float32)], 1), gr, h, v, pol)
        same_bits(ff.sum2(xd).cpu().numpy(), want)


@pytest.mark.parametrize("cond", [1e3, 1e6, 1e9, 1e12])
def test_dot2_ill_conditioned_within_bound(cond):
    import paper_cs_0603115_gb300 as ff
    n = 1 << 22
    g = inputs.ill_dot_f32(n, cond, inputs.seed_for(5, int(math.log10(cond))))
    x, y = g.x.to(DEV), g.y.to(DEV)
    r = ff.dot2(x, y).cpu().numpy()
    _, _, A, E = oracle.exact_dot_f32(g.x.numpy(), g.y.numpy(), r)
    grid, _, _ = _shape(x, y)
    u = 2.0 ** -24
    # s-additions along one path: the thread's own values, then the warp,
    # block and last-block trees; each adds at most u |p| of error terms
    m = -(-n // (grid * 256)) + 4 + 5 + 3 + (-(-grid // 256)) + 5 + 3
    gam = m * u / (1 - m * u)
    assert abs(E) <= gam * u * (m + 1) * A
    # and in practice at the level of u^2
    assert abs(E) <= 2.0 ** -40 * A
