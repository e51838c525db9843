"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds no float-float arithmetic: it only draws random binary64
values and stores each as a float-float pair (hi, lo) = (RN32(d), RN32(d - hi)),
the format of Section 4 of the paper (an unevaluated sum of two binary32
numbers).  The paper measured its operators on random inputs (Section 6.1);
the recipes below are the synthetic stand-ins.

Every generator takes a seed and a torch device.  The same seed on the same
device and torch version gives the same arrays; the CPU oracle and the CUDA
kernels always consume the same stored arrays (generated on the CPU and
copied, or generated on the GPU and sampled back), never two draws.

Shapes: a float-float vector of n values is a float32 tensor of shape
``(n, 2)``; a packed error-free-transformation input is ``(n, 2)`` of (a, b).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

SEED_BASE = 0xFF000000


def seed_for(config: int, stream: int) -> int:
    """Seed of input stream ``stream`` of workload ``config``."""
    return SEED_BASE + 16 * config + stream


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(seed)
    return g


def to_ff(d: torch.Tensor) -> torch.Tensor:
    """Store binary64 values as float-float pairs: hi = RN32(d), lo = RN32(d - hi).

    d - hi is exact in binary64, and hi + lo is exactly representable in
    binary64 (at most 49 significant bits), so the FP64 baselines can consume
    the exact value of every pair."""
    d = d.to(torch.float64)
    hi = d.to(torch.float32)
    lo = (d - hi.to(torch.float64)).to(torch.float32)
    return torch.stack([hi, lo], dim=-1).contiguous()


def ff_to_f64(x: torch.Tensor) -> torch.Tensor:
    """hi + lo in binary64 (exact for pairs made by ``to_ff``)."""
    return x[..., 0].to(torch.float64) + x[..., 1].to(torch.float64)


def loguniform_f64(n: int, g: torch.Generator, device, emin: float = -20.0,
                   emax: float = 20.0) -> torch.Tensor:
    """Random sign times 2^U, U uniform in [emin, emax]."""
    u = torch.rand(n, generator=g, dtype=torch.float64, device=device)
    s = torch.randint(0, 2, (n,), generator=g, device=device).to(torch.float64)
    return (2.0 * s - 1.0) * torch.exp2(emin + (emax - emin) * u)


@dataclass
class Elementwise:
    """Operands of the elementwise workloads.

    a, b      float-float (n, 2); 10% of b are -a (1 + u 2^-30) (cancellation)
    ab        packed binary32 pairs (a.hi, b.hi) for Add12 / Mul12
    a_sqrt    |a| (both components negated where a.hi < 0) for Sqrt22
    """
    a: torch.Tensor
    b: torch.Tensor
    ab: torch.Tensor
    a_sqrt: torch.Tensor


def elementwise(n: int, seed: int, device="cpu", cancel_frac: float = 0.1) -> Elementwise:
    """Magnitudes log-uniform over 2^-20 .. 2^20 with random signs; a fraction
    ``cancel_frac`` of the b values is set to -a (1 + u 2^-30), u in [0, 1),
    so that a + b cancels about 30 bits.  Divisors b satisfy |b| >= 2^-20 (1 -
    2^-30), far above the 2^-60 floor the operators assume."""
    g = _gen(seed, device)
    da = loguniform_f64(n, g, device)
    db = loguniform_f64(n, g, device)
    pick = torch.rand(n, generator=g, dtype=torch.float64, device=device) < cancel_frac
    u = torch.rand(n, generator=g, dtype=torch.float64, device=device)
    a = to_ff(da)
    av = ff_to_f64(a)
    db = torch.where(pick, -av * (1.0 + u * 2.0 ** -30), db)
    b = to_ff(db)
    ab = torch.stack([a[:, 0], b[:, 0]], dim=1).contiguous()
    neg = (a[:, 0] < 0).unsqueeze(1)
    a_sqrt = torch.where(neg, -a, a).contiguous()
    return Elementwise(a=a, b=b, ab=ab, a_sqrt=a_sqrt)


def _mant26(n: int, g: torch.Generator, device) -> torch.Tensor:
    """Random binary64 values m 2^-26 with a 26-bit integer m in [2^25, 2^26)
    and a random sign, i.e. |v| in [0.5, 1).  Products of two such values are
    exact in binary64."""
    m = torch.randint(2 ** 25, 2 ** 26, (n,), generator=g, device=device).to(torch.float64)
    s = torch.randint(0, 2, (n,), generator=g, device=device).to(torch.float64)
    return (2.0 * s - 1.0) * m * 2.0 ** -26


@dataclass
class IllDot:
    x: torch.Tensor          # (n, 2) float-float
    y: torch.Tensor          # (n, 2) float-float
    cond_target: float
    dot_design: float        # the binary64 value the construction aims at


def ill_dot(n: int, cond: float, seed: int, device="cpu") -> IllDot:
    """Ill-conditioned dot product with a prescribed condition number
    cond = 2 sum |x_i y_i| / |sum x_i y_i|, in the spirit of Ogita, Rump and
    Oishi's GenDot ("Accurate sum and dot product", 2005): terms spread over
    2^(2E) in magnitude with E = round(log2(cond) / 2), and massive cancellation.

    Vectorised construction (no sequential running dot):
      * the first half are free products x_i y_i, both factors with exponent
        e_i uniform in {0..E}, 26-bit significands and random signs;
      * each term of the second half cancels one free term (a random
        permutation) up to the binary64 rounding of y = -p / x;
      * the last term is set so that the whole sum is the design value
        T = 2 A / cond (A = the sum of the other |x_i y_i|, solved so that
        the final A, including the last term, gives cond);
      * the order is then randomly permuted.
    The stored pairs differ from the binary64 design by the float-float
    rounding of y (2^-48 relative); the achieved condition number is what the
    exact reference measures on the stored pairs.
    """
    if n < 4:
        raise ValueError("ill_dot needs n >= 4")
    g = _gen(seed, device)
    E = max(0, int(round(math.log2(cond) / 2)))
    h = n // 2
    m = n - h
    e1 = torch.randint(0, E + 1, (h,), generator=g, device=device).to(torch.float64)
    x1 = _mant26(h, g, device) * torch.exp2(e1)
    y1 = _mant26(h, g, device) * torch.exp2(e1)
    p1 = x1 * y1                                              # exact
    perm = torch.randperm(h, generator=g, device=device)
    if m > h:  # odd n: one more mirror term
        perm = torch.cat([perm, perm[:1]])
    e2 = torch.randint(0, E + 1, (m,), generator=g, device=device).to(torch.float64)
    x2 = _mant26(m, g, device) * torch.exp2(e2)
    y2 = -(p1[perm] / x2)
    x = torch.cat([x1, x2])
    y = torch.cat([y1, y2])
    xf = to_ff(x)
    yf = to_ff(y)
    # products of the stored pairs, as exact binary64 partial products
    xv = xf[:, 0].to(torch.float64)            # x has <= 26 bits: lo is exact
    xv = xv + xf[:, 1].to(torch.float64)
    prod_hi = xv * yf[:, 0].to(torch.float64)
    prod_lo = xv * yf[:, 1].to(torch.float64)
    rest_s = (prod_hi[:-1].sum() + prod_lo[:-1].sum()).item()
    rest_a = (prod_hi[:-1] + prod_lo[:-1]).abs().sum().item()
    # |T| solving 2 (A_rest + |T - S_rest|) / |T| = cond, sign of T = sign(S_rest)
    sgn = 1.0 if rest_s >= 0 else -1.0
    t_abs = 2.0 * (rest_a - abs(rest_s)) / (cond - 2.0) if cond > 2 else abs(rest_s) + rest_a
    if t_abs < abs(rest_s):
        t_abs = 2.0 * (rest_a + abs(rest_s)) / (cond + 2.0)
    T = sgn * t_abs
    need = T - rest_s
    el = max(0, int(round(math.log2(abs(need)) / 2))) if need != 0 else 0
    x_last = (_mant26(1, g, device) * 2.0 ** el)[0]
    x = x.clone()
    x[-1] = x_last
    y = y.clone()
    y[-1] = need / x_last
    xf = to_ff(x)
    yf = to_ff(y)
    order = torch.randperm(n, generator=g, device=device)
    return IllDot(x=xf[order].contiguous(), y=yf[order].contiguous(),
                  cond_target=float(cond), dot_design=float(T))


def _mant24(n: int, g: torch.Generator, device) -> torch.Tensor:
    """Random binary32-representable values with 24-bit significands in
    [0.5, 1) and random signs (as binary64)."""
    m = torch.randint(2 ** 23, 2 ** 24, (n,), generator=g, device=device).to(torch.float64)
    s = torch.randint(0, 2, (n,), generator=g, device=device).to(torch.float64)
    return (2.0 * s - 1.0) * m * 2.0 ** -24


@dataclass
class IllDotF32:
    x: torch.Tensor          # (n,) binary32
    y: torch.Tensor          # (n,) binary32
    cond_target: float
    dot_design: float


def ill_dot_f32(n: int, cond: float, seed: int, device="cpu") -> IllDotF32:
    """The ill-conditioned dot of ``ill_dot`` for plain binary32 vectors (the
    inputs of the compensated Sum2 / Dot2): same construction, every value a
    binary32 number, so every product x_i y_i is exact in binary64 and the
    design sum is formed from exact products."""
    if n < 4:
        raise ValueError("ill_dot_f32 needs n >= 4")
    g = _gen(seed, device)
    E = max(0, int(round(math.log2(cond) / 2)))
    h = n // 2
    m = n - h
    e1 = torch.randint(0, E + 1, (h,), generator=g, device=device).to(torch.float64)
    x1 = _mant24(h, g, device) * torch.exp2(e1)
    y1 = _mant24(h, g, device) * torch.exp2(e1)
    p1 = x1 * y1
    perm = torch.randperm(h, generator=g, device=device)
    if m > h:
        perm = torch.cat([perm, perm[:1]])
    e2 = torch.randint(0, E + 1, (m,), generator=g, device=device).to(torch.float64)
    x2 = _mant24(m, g, device) * torch.exp2(e2)
    y2 = (-(p1[perm] / x2)).to(torch.float32).to(torch.float64)
    x = torch.cat([x1, x2])
    y = torch.cat([y1, y2])
    prod = x * y                                              # exact
    rest_s = prod[:-1].sum().item()
    rest_a = prod[:-1].abs().sum().item()
    sgn = 1.0 if rest_s >= 0 else -1.0
    t_abs = 2.0 * (rest_a - abs(rest_s)) / (cond - 2.0) if cond > 2 else abs(rest_s) + rest_a
    if t_abs < abs(rest_s):
        t_abs = 2.0 * (rest_a + abs(rest_s)) / (cond + 2.0)
    T = sgn * t_abs
    need = T - rest_s
    el = max(0, int(round(math.log2(abs(need)) / 2))) if need != 0 else 0
    x_last = (_mant24(1, g, device) * 2.0 ** el)[0]
    x = x.clone()
    y = y.clone()
    x[-1] = x_last
    y[-1] = float(torch.tensor(need / float(x_last), dtype=torch.float64).to(torch.float32))
    order = torch.randperm(n, generator=g, device=device)
    return IllDotF32(x=x[order].to(torch.float32).contiguous(), y=y[order].to(torch.float32).contiguous(),
                     cond_target=float(cond), dot_design=float(T))


@dataclass
class GemvInputs:
    A: torch.Tensor   # (m, n, 2) row-major float-float
    X: torch.Tensor   # (k, n, 2): column c of X is X[c]  (n x k column-major)
    dY: torch.Tensor  # (k, m, 2): column c of dY is dY[c] (m x k column-major)


def gemv(m: int, n: int, k: int, seed: int, device="cpu") -> GemvInputs:
    """A, X and dY with the elementwise magnitude law (no forced cancellation)."""
    g = _gen(seed, device)
    A = to_ff(loguniform_f64(m * n, g, device)).reshape(m, n, 2)
    X = to_ff(loguniform_f64(k * n, g, device)).reshape(k, n, 2)
    dY = to_ff(loguniform_f64(k * m, g, device)).reshape(k, m, 2)
    return GemvInputs(A=A, X=X, dY=dY)


@dataclass
class GemmInputs:
    A: torch.Tensor   # (m, kk, 2)
    B: torch.Tensor   # (kk, n, 2)
    dC: torch.Tensor  # (m, n, 2)


def gemm(m: int, n: int, kk: int, seed: int, device="cpu") -> GemmInputs:
    """Row-major A (m x kk), B (kk x n) and an output gradient dC (m x n), all
    with the elementwise magnitude law (no forced cancellation)."""
    g = _gen(seed, device)
    A = to_ff(loguniform_f64(m * kk, g, device)).reshape(m, kk, 2)
    B = to_ff(loguniform_f64(kk * n, g, device)).reshape(kk, n, 2)
    dC = to_ff(loguniform_f64(m * n, g, device)).reshape(m, n, 2)
    return GemmInputs(A=A, B=B, dC=dC)


def batch_lengths(count: int, seed: int, lo_exp: float = 2.0, hi_exp: float = 7.0):
    """Instance lengths round(10^(lo + (hi - lo) u)), u uniform, and kinds: half
    dot (0), half AXPY (1), assigned by a seeded shuffle."""
    g = _gen(seed, "cpu")
    u = torch.rand(count, generator=g, dtype=torch.float64)
    lengths = torch.round(10.0 ** (lo_exp + (hi_exp - lo_exp) * u)).to(torch.int64)
    kinds = torch.tensor([i % 2 for i in range(count)], dtype=torch.int32)
    kinds = kinds[torch.randperm(count, generator=g)]
    return lengths.tolist(), kinds.tolist()


def scalar_ff(seed: int) -> torch.Tensor:
    """One float-float scalar with the elementwise magnitude law (CPU)."""
    g = _gen(seed, "cpu")
    return to_ff(loguniform_f64(1, g, "cpu"))[0]
