"""Pins of the CPU oracle to what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks an algorithm
against a theorem of Section 4.1 (exactness of Add12 and Mul12, the Split
non-overlap, the Add22 and Mul22 bounds), against an independent exact
reference (the superaccumulator, binary128, Python fractions, numpy's own
binary32 arithmetic), against closed forms, or against special cases that
reduce one operator to another.  A dropped term, a wrong sign or a
transposed operand in any operator makes at least one of them fail.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

from paper_cs_0603115_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
f32 = np.float32


def ff(*pairs):
    return np.array(pairs, dtype=np.float32).reshape(-1, 2)


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


def assert_same_up_to_zero_sign(x, y):
    """Bitwise equal, except that a zero may carry either sign.  The pair
    (RN(ab), ab - RN(ab)) is unique as a pair of values; the fused form
    returns +0 for an exact product, Dekker's form may return -0."""
    x = np.asarray(x, np.float32); y = np.asarray(y, np.float32)
    assert np.all(x == y)
    nz = x != 0
    np.testing.assert_array_equal(bits(x[nz]), bits(y[nz]))


def sig_bits(v):
    """Number of significant bits of each binary32 value (0 for zero)."""
    v = np.asarray(v, dtype=np.float32)
    u = v.view(np.uint32).astype(np.int64)
    exp = (u >> 23) & 0xFF
    man = u & 0x7FFFFF
    man = np.where(exp > 0, man | 0x800000, man)
    out = np.zeros(v.shape, dtype=np.int64)
    nz = man != 0
    m = man[nz]
    tz = np.zeros(m.shape, dtype=np.int64)
    mm = m.copy()
    while True:
        even = (mm & 1) == 0
        if not even.any():
            break
        tz += even
        mm = np.where(even, mm >> 1, mm)
    width = np.floor(np.log2(m)).astype(np.int64) + 1
    out[nz] = width - tz
    return out


def subset_floats():
    """A small float subset for brute force: both signs, exponents -30..30
    step 3, extreme significands (0x800000..0x80000F, 0xFFFFF0..0xFFFFFF) and
    1, 3, 4097, 2^12 - 1, 2^12 + 1."""
    mants = list(range(0x800000, 0x800010)) + list(range(0xFFFFF0, 0x1000000))
    base = [m * 2.0 ** -23 for m in mants] + [1.0, 3.0, 4097.0, 4095.0, 4097.0 / 2]
    vals = []
    for e in range(-30, 31, 3):
        for m in base:
            for s in (1.0, -1.0):
                vals.append(s * m * 2.0 ** e)
    return np.unique(np.array(vals, dtype=np.float32))


def all_pairs(S):
    a, b = np.meshgrid(S, S, indexing="ij")
    return np.stack([a.ravel(), b.ravel()], axis=1).astype(np.float32)


# --------------------------------------------------------------------------
# build canaries
# --------------------------------------------------------------------------

def test_no_contraction_canary(orc):
    # (1 + 2^-12)^2 = 1 + 2^-11 + 2^-24; RN32 of it ties to 1 + 2^-11, so the
    # unfused a*b + c is exactly 0 while a fused one gives 2^-24.
    a = 1 + 2.0 ** -12
    c = -(1 + 2.0 ** -11)
    assert orc.canary_mul_add(a, a, c) == 0.0
    assert float(np.fma(f32(a), f32(a), f32(c))) == 2.0 ** -24 if hasattr(np, "fma") else True


def test_subnormals_kept(orc):
    a, b = 2.0 ** -140, 2.0 ** -149
    se = orc.add12(ff(a, b))
    assert se[0, 0] == f32(a) + f32(b) and se[0, 0] != 0 and se[0, 1] == 0
    p = orc.mul12(ff(2.0 ** -70, 2.0 ** -70))   # product 2^-140 is subnormal
    assert p[0, 0] == f32(2.0 ** -140)


# --------------------------------------------------------------------------
# Add12 (Add12 theorem): s = RN(a + b), s + r = a + b exactly
# --------------------------------------------------------------------------

def test_add12_bruteforce_exact(orc):
    ab = all_pairs(subset_floats())
    se = orc.add12(ab)
    assert orc.count_sum2_mismatch(ab, se) == 0
    np.testing.assert_array_equal(bits(se[:, 0]), bits(ab[:, 0] + ab[:, 1]))
    assert np.all(np.abs(se[:, 1]) <= np.spacing(np.abs(se[:, 0])) / 2)


def test_add12_random_wide_exponents_exact(orc):
    rng = np.random.default_rng(1)
    n = 200000
    e = rng.integers(-120, 120, size=(n, 2))
    m = rng.uniform(1, 2, size=(n, 2)) * rng.choice([-1, 1], size=(n, 2))
    ab = (m * 2.0 ** e).astype(np.float32)
    se = orc.add12(ab)
    assert orc.count_sum2_mismatch(ab, se) == 0
    np.testing.assert_array_equal(bits(se[:, 0]), bits(ab[:, 0] + ab[:, 1]))


def test_add12_paper_anomaly_is_exact_under_rn(orc):
    # The paper's Table 5 reports an Add12 error of 2^-48 on its GPU for
    # operands of opposite signs whose significands do not overlap; under
    # IEEE round-to-nearest the Add12 theorem makes those cases exact.
    gold = json.load(open(os.path.join(GOLDEN, "paper_accuracy.json")))
    assert gold["max_error_log2"]["Add12"] == -48.0
    ab = ff((1.0, -2.0 ** -30), (2.0 ** 20, -(2.0 ** -10 + 2.0 ** -20)),
            (-3.0, 2.0 ** -40), (1.5, -1.5 * 2.0 ** -25), (2.0 ** 24, -1.0),
            (1.0, -2.0 ** -24), (1.0, -2.0 ** -25), (-1.0, 2.0 ** -24 * 3))
    se = orc.add12(ab)
    assert orc.count_sum2_mismatch(ab, se) == 0


# --------------------------------------------------------------------------
# Split (Split theorem), s = 12
# --------------------------------------------------------------------------

def test_split_nonoverlap_and_exact(orc):
    S = subset_floats()
    # the "every significand bit set except the last two" cases of the proof
    special = [m * 2.0 ** -23 * 2.0 ** e for m in range(0xFFFFFC, 0x1000000)
               for e in range(-20, 21, 5)]
    a = np.concatenate([S, np.array(special, np.float32), -np.array(special, np.float32)])
    hl = orc.split(a)
    hi, lo = hl[:, 0], hl[:, 1]
    # a = hi + lo exactly (both binary32 with nearby exponents: exact in f64)
    np.testing.assert_array_equal(hi.astype(np.float64) + lo.astype(np.float64), a.astype(np.float64))
    assert np.all(sig_bits(hi) <= 12)
    assert np.all(sig_bits(lo) <= 12)
    assert np.all(np.abs(hi) >= np.abs(lo))


def test_split_matches_fractions(orc):
    a = np.array([1.0, 0.1, 3.14159265, -2.718281828, 12345.678], np.float32)
    hl = orc.split(a)
    for v, (h, l) in zip(a, hl):
        assert Fraction(float(h)) + Fraction(float(l)) == Fraction(float(v))


# --------------------------------------------------------------------------
# Mul12 (Mul12 theorem): x = RN(ab), x + y = ab exactly; Dekker == fused
# --------------------------------------------------------------------------

def test_mul12_bruteforce_exact_and_forms_agree(orc):
    ab = all_pairs(subset_floats())
    xy = orc.mul12(ab)
    xd = orc.mul12_dekker(ab)
    assert orc.count_prod_mismatch(ab, xy) == 0
    assert orc.count_prod_mismatch(ab, xd) == 0
    assert_same_up_to_zero_sign(xy, xd)
    np.testing.assert_array_equal(bits(xy[:, 0]), bits(ab[:, 0] * ab[:, 1]))
    # exact in binary64 too: a*b has at most 48 bits
    np.testing.assert_array_equal(xy[:, 0].astype(np.float64) + xy[:, 1],
                                  ab[:, 0].astype(np.float64) * ab[:, 1])


def test_mul12_random_domain(orc):
    # domain of the theorem: no underflow of the error term (|ab| >= 2^-100)
    # and no overflow
    rng = np.random.default_rng(2)
    n = 200000
    e = rng.integers(-50, 50, size=(n, 2))
    m = rng.uniform(1, 2, size=(n, 2)) * rng.choice([-1, 1], size=(n, 2))
    ab = (m * 2.0 ** e).astype(np.float32)
    xy = orc.mul12(ab)
    assert orc.count_prod_mismatch(ab, xy) == 0
    assert_same_up_to_zero_sign(xy, orc.mul12_dekker(ab))


# --------------------------------------------------------------------------
# float-float operand sets
# --------------------------------------------------------------------------

def ff_subset():
    """Float-float values (hi, lo) with hi from a subset and lo in
    {0, +-0.75 ulp-scale, +-2^-30 hi}."""
    S = subset_floats()[::4]
    out = []
    for h in S:
        h = float(h)
        for lo in (0.0, h * 2.0 ** -25 * 1.5, -h * 2.0 ** -25 * 1.25, h * 2.0 ** -30, -h * 2.0 ** -33):
            l32 = f32(lo)
            # keep (hi, lo) normalised: |lo| <= ulp(hi) / 2
            if abs(float(l32)) <= float(np.spacing(f32(abs(h)))) / 2:
                out.append((h, float(l32)))
    return np.array(out, np.float32)


def rand_ff(n, seed, cancel=0.1):
    e = inputs.elementwise(n, seed, cancel_frac=cancel)
    return e.a.numpy(), e.b.numpy(), e.a_sqrt.numpy()


# --------------------------------------------------------------------------
# Add22 (Add22 theorem)
# --------------------------------------------------------------------------

def _check_add22_bound(orc, a, b):
    r = orc.add22(a, b)
    bd = orc.add22_bound(a, b, r)
    bound = np.maximum(bd[:, 1], bd[:, 2])
    return int(np.sum(bd[:, 0] > bound))


def test_add22_bound_random(orc):
    a, b, _ = rand_ff(1 << 17, inputs.seed_for(0, 5))
    assert _check_add22_bound(orc, a, b) == 0


def test_add22_bound_bruteforce(orc):
    F = ff_subset()
    idx = np.random.default_rng(3).choice(F.shape[0], size=(400000, 2))
    assert _check_add22_bound(orc, F[idx[:, 0]], F[idx[:, 1]]) == 0


def test_add22_reduces_to_add12(orc):
    S = subset_floats()
    ab = all_pairs(S[::2])
    a = np.stack([ab[:, 0], np.zeros(len(ab), np.float32)], 1)
    b = np.stack([ab[:, 1], np.zeros(len(ab), np.float32)], 1)
    r = orc.add22(a, b)
    se = orc.add12(ab)
    np.testing.assert_array_equal(r, se)


def test_add22_closed_forms(orc):
    # (1, 2^-30) + (2^-10, 2^-40) = 1 + 2^-10 + 2^-30 + 2^-40: hi = 1 + 2^-10,
    # lo = 2^-30 + 2^-40 (fits in 24 bits)
    r = orc.add22(ff(1.0, 2.0 ** -30), ff(2.0 ** -10, 2.0 ** -40))
    assert r[0, 0] == f32(1 + 2.0 ** -10) and r[0, 1] == f32(2.0 ** -30 + 2.0 ** -40)
    # cancellation of the high parts leaves the sum of the low parts
    r = orc.add22(ff(1.0, 2.0 ** -30), ff(-1.0, 2.0 ** -31))
    assert r[0, 0] == f32(1.5 * 2.0 ** -30) and r[0, 1] == 0
    # tie |ah| == |bh| with the same sign
    r = orc.add22(ff(1.0, 2.0 ** -26), ff(1.0, -2.0 ** -27))
    assert float(r[0, 0]) + float(r[0, 1]) == 2 + 2.0 ** -27


def add22_low_part_order_cases():
    """Worked examples, derived by hand, in which the order of the two low
    parts in Add22's s (Section 4.1, Add22 theorem: the low part of the
    operand with the smaller high part is added first, then the other one)
    decides the result.

    a = (2^24, 2^-24 + 2^-47), b = (1, 2^-24): |ah| >= |bh|, r = RN(2^24 + 1)
    = 2^24 (a tie, to even), ah - r = 0, + bh = 1, then
      paper order   + bl = RN(1 + 2^-24) = 1 (tie, to even),
                    + al = RN(1 + 2^-24 + 2^-47) = 1 + 2^-23  -> s = 1 + 2^-23
      swapped order + al = 1 + 2^-23, + bl = RN(1 + 2^-23 + 2^-24)
                    = 1 + 2^-22 (tie, to even)                -> s = 1 + 2^-22
    and Add12(r, s) = (RN(2^24 + s), 2^24 + s - RN(2^24 + s)):
      paper order   (2^24 + 2, -1 + 2^-23); swapped (2^24 + 2, -1 + 2^-22).
    Exchanging a and b takes the other branch with the same operands in the
    same roles, so both branches must give the first pair.  Scaling every
    part by 2^e (no under- or overflow) and negating every part scale and
    negate the result exactly."""
    cases = []
    for e in (-20, 0, 20):
        for sgn in (1.0, -1.0):
            k = sgn * 2.0 ** e
            a = (k * 2.0 ** 24, k * (2.0 ** -24 + 2.0 ** -47))
            b = (k * 1.0, k * 2.0 ** -24)
            want = (k * (2.0 ** 24 + 2), k * (-1 + 2.0 ** -23))
            cases.append((a, b, want))   # first branch  (|ah| >= |bh|)
            cases.append((b, a, want))   # second branch (|ah| <  |bh|)
    a = np.array([c[0] for c in cases], np.float32)
    b = np.array([c[1] for c in cases], np.float32)
    want = np.array([c[2] for c in cases], np.float32)
    # every constant above is a binary32 value (no rounding on the way in)
    for arr, src in ((a, [c[0] for c in cases]), (b, [c[1] for c in cases]), (want, [c[2] for c in cases])):
        assert np.array_equal(arr.astype(np.float64), np.array(src, np.float64))
    return a, b, want


def test_add22_low_part_order(orc):
    a, b, want = add22_low_part_order_cases()
    np.testing.assert_array_equal(bits(orc.add22(a, b)), bits(want))


def test_add22_geometric_series_sum(orc):
    # sum_{i=0}^{40} 2^-i = 2 - 2^-40 = (2, -2^-40) exactly
    x = np.stack([2.0 ** -np.arange(41), np.zeros(41)], 1).astype(np.float32)
    s = orc.ff_sum(x)
    assert s[0] == 2.0 and s[1] == f32(-(2.0 ** -40))


# --------------------------------------------------------------------------
# Mul22 (Mul22 theorem): relative error <= 2^-44
# --------------------------------------------------------------------------

def test_mul22_bound_random(orc):
    a, b, _ = rand_ff(1 << 17, inputs.seed_for(0, 6))
    r = orc.mul22(a, b)
    re = orc.relerr("mul", a, b, r)
    assert re.max() <= 2.0 ** -44
    gold = json.load(open(os.path.join(GOLDEN, "paper_accuracy.json")))
    assert math.log2(re.max()) <= gold["max_error_log2"]["Mul22"] + 1.0


def test_mul22_bound_bruteforce(orc):
    F = ff_subset()
    idx = np.random.default_rng(4).choice(F.shape[0], size=(400000, 2))
    a, b = F[idx[:, 0]], F[idx[:, 1]]
    r = orc.mul22(a, b)
    assert orc.relerr("mul", a, b, r).max() <= 2.0 ** -44
    assert_same_up_to_zero_sign(r, orc.mul22_dekker(a, b))


def test_mul22_reduces_to_mul12(orc):
    ab = all_pairs(subset_floats()[::2])
    z = np.zeros(len(ab), np.float32)
    r = orc.mul22(np.stack([ab[:, 0], z], 1), np.stack([ab[:, 1], z], 1))
    xy = orc.mul12(ab)
    assert np.all(r == xy)


def test_mul22_closed_forms(orc):
    # (1 + 2^-30)^2 = 1 + 2^-29 + 2^-60; Mul22 drops al*bl = 2^-60
    r = orc.mul22(ff(1.0, 2.0 ** -30), ff(1.0, 2.0 ** -30))
    assert r[0, 0] == 1.0 and r[0, 1] == f32(2.0 ** -29)
    # (1 + 2^-20)^2 = 1 + 2^-19 + 2^-40 exactly
    r = orc.mul22(ff(1 + 2.0 ** -20, 0.0), ff(1 + 2.0 ** -20, 0.0))
    assert r[0, 0] == f32(1 + 2.0 ** -19) and r[0, 1] == f32(2.0 ** -40)
    # (3, 0) * (1, 2^-30): the al/bl cross term must enter: 3 + 3 2^-30
    r = orc.mul22(ff(3.0, 0.0), ff(1.0, 2.0 ** -30))
    assert r[0, 0] == 3.0 and r[0, 1] == f32(3 * 2.0 ** -30)
    r = orc.mul22(ff(1.0, 2.0 ** -30), ff(3.0, 0.0))
    assert r[0, 0] == 3.0 and r[0, 1] == f32(3 * 2.0 ** -30)


# --------------------------------------------------------------------------
# Div22 and Sqrt22 (Dekker's div2 / sqrt2)
# --------------------------------------------------------------------------

def test_div22_special_cases(orc):
    r = orc.div22(ff(6.0, 0.0), ff(3.0, 0.0))
    assert r[0, 0] == 2.0 and r[0, 1] == 0
    r = orc.div22(ff(3.0, 3 * 2.0 ** -30), ff(3.0, 0.0))
    assert r[0, 0] == 1.0 and r[0, 1] == f32(2.0 ** -30)
    # (1 + 2^-19 + 2^-40) / (1 + 2^-20) = 1 + 2^-20 exactly
    r = orc.div22(ff(1 + 2.0 ** -19, 2.0 ** -40), ff(1 + 2.0 ** -20, 0.0))
    assert r[0, 0] == f32(1 + 2.0 ** -20) and r[0, 1] == 0
    a, b, _ = rand_ff(4096, inputs.seed_for(0, 7))
    one = np.tile(ff(1.0, 0.0), (len(a), 1))
    np.testing.assert_array_equal(orc.div22(a, one), orc.add12(a))
    q = orc.div22(a, a)
    assert np.all(q[:, 0] == 1.0) and np.all(q[:, 1] == 0)


def test_div22_accuracy(orc):
    a, b, _ = rand_ff(1 << 17, inputs.seed_for(0, 8))
    r = orc.div22(a, b)
    assert orc.relerr("div", a, b, r).max() <= 2.0 ** -43


def test_div22_sqrt22_bruteforce(orc):
    """Every ordered pair of the float-float subset (extreme significands,
    exponents -30..30, low parts 0, about ulp/2 and 2^-30 hi): Div22 within
    2^-44 of the exact quotient, and Sqrt22 of every subset value (made
    non-negative) within 2^-44 of the exact square root (binary128)."""
    F = ff_subset()
    i, j = np.meshgrid(np.arange(F.shape[0]), np.arange(F.shape[0]), indexing="ij")
    a, b = F[i.ravel()], F[j.ravel()]
    r = orc.div22(a, b)
    assert orc.relerr("div", a, b, r).max() <= 2.0 ** -44
    s = F.copy()
    s[s[:, 0] < 0] *= -1
    assert orc.relerr("sqrt", s, None, orc.sqrt22(s)).max() <= 2.0 ** -44


def test_sqrt22_special_cases(orc):
    r = orc.sqrt22(ff((4.0, 0.0), (0.0, 0.0), (-0.0, 0.0), (-1.0, 0.0),
                      (1 + 2.0 ** -19, 2.0 ** -40), (9.0, 0.0), (2.0 ** -40, 0.0)))
    assert r[0, 0] == 2 and r[0, 1] == 0
    assert r[1, 0] == 0 and not np.signbit(r[1, 0])
    assert r[2, 0] == 0 and np.signbit(r[2, 0])
    assert np.isnan(r[3]).all()
    assert r[4, 0] == f32(1 + 2.0 ** -20) and r[4, 1] == 0
    assert r[5, 0] == 3 and r[5, 1] == 0
    assert r[6, 0] == f32(2.0 ** -20) and r[6, 1] == 0


def test_sqrt22_accuracy_and_square_roundtrip(orc):
    _, _, a = rand_ff(1 << 17, inputs.seed_for(0, 9))
    r = orc.sqrt22(a)
    assert orc.relerr("sqrt", a, None, r).max() <= 2.0 ** -43
    sq = orc.mul22(r, r)
    assert orc.relerr("add", sq, np.zeros_like(sq), a).max() < 2.0 ** -42


# --------------------------------------------------------------------------
# exact references: the superaccumulator and binary128
# --------------------------------------------------------------------------

def test_superaccumulator_matches_fsum(orc):
    rng = np.random.default_rng(5)
    for trial in range(20):
        n = int(rng.integers(1, 5000))
        v = rng.standard_normal(n) * 2.0 ** rng.integers(-1000, 1000, n)
        v = np.concatenate([v, -v[: n // 2] * (1 + 2.0 ** -50), [2.0 ** -1074, 5e-324]])
        assert orc.exact_sum_f64(v) == math.fsum(v.tolist())


def test_superaccumulator_binary128_vs_fractions(orc):
    rng = np.random.default_rng(6)
    for trial in range(20):
        v = rng.standard_normal(50) * 2.0 ** rng.integers(-60, 60, 50)
        exact = sum(Fraction(float(t)) for t in v)
        hi, lo = orc.exact_sum_f64_q(v)
        got = Fraction(hi) + Fraction(lo)
        if exact == 0:
            assert got == 0
        else:
            assert abs(got - exact) <= abs(exact) * Fraction(1, 2 ** 105)


def test_relerr_reference_vs_fractions(orc):
    a, b, asq = rand_ff(64, inputs.seed_for(0, 10))
    val = lambda p: Fraction(float(p[0])) + Fraction(float(p[1]))
    for op, fn, exact in (("add", orc.add22, lambda x, y: val(x) + val(y)),
                          ("mul", orc.mul22, lambda x, y: val(x) * val(y)),
                          ("div", orc.div22, lambda x, y: val(x) / val(y))):
        r = fn(a, b)
        re = orc.relerr(op, a, b, r)
        for i in range(len(a)):
            ex = exact(a[i], b[i])
            want = abs((val(r[i]) - ex) / ex) if ex != 0 else abs(val(r[i]))
            assert abs(Fraction(re[i]) - want) <= want * Fraction(1, 2 ** 40) + Fraction(1, 2 ** 200)


# --------------------------------------------------------------------------
# reductions, AXPY, backward, GEMV
# --------------------------------------------------------------------------

def test_sum_of_ones(orc):
    for n in (1, 2, 3, 1000, 12345):
        s = orc.ff_sum(np.tile(ff(1.0, 0.0), (n, 1)))
        assert s[0] == n and s[1] == 0


def test_dot_with_ones_is_sum_and_n1_is_mul22(orc):
    a, b, _ = rand_ff(5000, inputs.seed_for(0, 11))
    one = np.tile(ff(1.0, 0.0), (len(a), 1))
    np.testing.assert_array_equal(orc.ff_dot(a, one), orc.ff_sum(a))
    np.testing.assert_array_equal(orc.ff_dot(a[:1], b[:1]), orc.mul22(a[:1], b[:1])[0])
    z = orc.ff_dot(a[:0], b[:0])
    assert z[0] == 0 and z[1] == 0


@pytest.mark.parametrize("cond", [1e3, 1e6, 1e9, 1e12])
def test_dot_ill_conditioned_within_bound(orc, cond):
    g = inputs.ill_dot(1 << 16, cond, inputs.seed_for(2, 1))
    x, y = g.x.numpy(), g.y.numpy()
    res = orc.ff_dot(x, y)
    s_hi, s_lo, A, E = orc.exact_dot(x, y, res)
    achieved = 2 * A / abs(s_hi)
    assert 0.5 * cond <= achieved <= 2 * cond
    n = x.shape[0]
    # per-step Add22 error <= 2^-44 (|acc| + |term|) gives n 2^-44 sum|x_i y_i|
    assert abs(E) <= n * 2.0 ** -44 * A


def test_axpy_special_cases(orc):
    a, b, _ = rand_ff(4096, inputs.seed_for(0, 12))
    one = ff(1.0, 0.0)[0]
    np.testing.assert_array_equal(orc.axpy(one, a, b), orc.add22(a, b))
    z = orc.axpy(ff(3.0, 0.0)[0], a, np.zeros_like(a))
    np.testing.assert_array_equal(z, orc.mul22(np.tile(ff(3.0, 0.0), (len(a), 1)), a))


def test_dot_backward_accuracy(orc):
    a, b, _ = rand_ff(4096, inputs.seed_for(0, 13))
    dout = ff(1.0 / 3.0, f32(1.0 / 3.0 - float(f32(1.0 / 3.0))))[0]
    dx, dy = orc.dot_backward(dout, a, b)
    D = np.tile(dout, (len(a), 1))
    assert orc.relerr("mul", D, b, dx).max() <= 2.0 ** -44
    assert orc.relerr("mul", D, a, dy).max() <= 2.0 ** -44
    dx1, dy1 = orc.dot_backward(ff(1.0, 0.0)[0], a, b)
    np.testing.assert_array_equal(dx1, orc.add12(b))
    np.testing.assert_array_equal(dy1, orc.add12(a))


def test_gemv_identity_and_transpose(orc):
    m = n = 24
    k = 3
    gi = inputs.gemv(m, n, k, inputs.seed_for(4, 1))
    A, X, dY = gi.A.numpy(), gi.X.numpy(), gi.dY.numpy()
    I = np.zeros((n, n, 2), np.float32)
    I[np.arange(n), np.arange(n), 0] = 1.0
    np.testing.assert_array_equal(orc.gemv(I, X), orc.add12(X.reshape(-1, 2)).reshape(X.shape))
    np.testing.assert_array_equal(orc.gemv_t(I, X), orc.add12(X.reshape(-1, 2)).reshape(X.shape))
    # A^T dY computed by gemv_t equals gemv on the explicit transpose
    At = np.ascontiguousarray(A.transpose(1, 0, 2))
    np.testing.assert_array_equal(orc.gemv_t(A, dY), orc.gemv(At, dY))


def test_gemv_rows_within_bound(orc):
    m, n, k = 16, 300, 2
    gi = inputs.gemv(m, n, k, inputs.seed_for(4, 2))
    A, X = gi.A.numpy(), gi.X.numpy()
    Y = orc.gemv(A, X)
    for c in range(k):
        for r in range(m):
            s_hi, s_lo, Aabs, E = orc.exact_dot(A[r], X[c], Y[c, r])
            assert abs(E) <= n * 2.0 ** -44 * Aabs
    # a single nonzero column of X picks out one column of A
    Xe = np.zeros((1, n, 2), np.float32)
    Xe[0, 7, 0] = 1.0
    np.testing.assert_array_equal(orc.gemv(A, Xe)[0], orc.add12(A[:, 7]))


def test_generator_hits_condition_numbers(orc):
    for cond in (1e3, 1e12):
        g = inputs.ill_dot(4096, cond, 77)
        s_hi, s_lo, A, E = orc.exact_dot(g.x.numpy(), g.y.numpy())
        assert 0.9 * cond <= 2 * A / abs(s_hi) <= 1.1 * cond


def test_fp32_baselines(orc):
    rng = np.random.default_rng(8)
    a, b, c = (rng.standard_normal(1000).astype(np.float32) for _ in range(3))
    np.testing.assert_array_equal(orc.fp32_add(a, b), a + b)
    np.testing.assert_array_equal(orc.fp32_mul(a, b), a * b)
    np.testing.assert_array_equal(orc.fp32_mad(a, b, c), (a * b) + c)


# --------------------------------------------------------------------------
# accurate addition (Joldes-Muller-Popescu Algorithm 6): no cancellation term
# --------------------------------------------------------------------------
U24 = 2.0 ** -24
ACC_ADD_BOUND = 3 * U24 * U24 / (1 - 4 * U24)


def test_add22_accurate_bound_random_with_cancellation(orc):
    a, b, _ = rand_ff(1 << 17, inputs.seed_for(0, 14), cancel=0.3)
    r = orc.add22_accurate(a, b)
    re = orc.relerr("add", a, b, r)
    assert re.max() <= ACC_ADD_BOUND
    # the paper's Add22 exceeds it by orders of magnitude on the same inputs
    assert orc.relerr("add", a, b, orc.add22(a, b)).max() > 2.0 ** -30


def test_add22_accurate_bruteforce(orc):
    F = ff_subset()
    idx = np.random.default_rng(9).choice(F.shape[0], size=(400000, 2))
    a, b = F[idx[:, 0]], F[idx[:, 1]]
    assert orc.relerr("add", a, b, orc.add22_accurate(a, b)).max() <= ACC_ADD_BOUND


def test_add22_accurate_special_cases(orc):
    ab = all_pairs(subset_floats()[::2])
    z = np.zeros(len(ab), np.float32)
    r = orc.add22_accurate(np.stack([ab[:, 0], z], 1), np.stack([ab[:, 1], z], 1))
    assert np.all(r == orc.add12(ab))
    r = orc.add22_accurate(ff(1.0, 2.0 ** -30), ff(-1.0, 2.0 ** -31))
    assert r[0, 0] == f32(1.5 * 2.0 ** -30) and r[0, 1] == 0
    # cancellation that Add22 gets wrong: (1, 2^-25) + (-(1 - 2^-24), -2^-48)
    a, b = ff(1.0, 2.0 ** -25), ff(-(1 - 2.0 ** -24), -(2.0 ** -48))
    r = orc.add22_accurate(a, b)
    want = Fraction(1) + Fraction(1, 2 ** 25) - (1 - Fraction(1, 2 ** 24)) - Fraction(1, 2 ** 48)
    got = Fraction(float(r[0, 0])) + Fraction(float(r[0, 1]))
    assert abs(got - want) <= abs(want) * Fraction(ACC_ADD_BOUND)


# --------------------------------------------------------------------------
# Sum2 / Dot2 (Ogita-Rump-Oishi) on binary32 vectors
# --------------------------------------------------------------------------

def gamma(n):
    return n * U24 / (1 - n * U24)


@pytest.mark.parametrize("cond", [1e3, 1e8, 1e12])
def test_dot2_within_oro_bound_small_n(orc, cond):
    # n small enough that gamma_n^2 << u: a dropped error term would show
    for seed in range(20):
        g = inputs.ill_dot_f32(32, cond, inputs.seed_for(5, seed))
        x, y = g.x.numpy(), g.y.numpy()
        r = orc.dot2(x, y)
        _, _, A, E = orc.exact_dot_f32(x, y, r)
        assert abs(E) <= gamma(32) ** 2 * A


def test_sum2_within_oro_bound_and_exact_cases(orc):
    rng = np.random.default_rng(10)
    for _ in range(20):
        x = (rng.standard_normal(48) * 2.0 ** rng.integers(-20, 20, 48)).astype(np.float32)
        x = np.concatenate([x, -x[:24] * np.float32(1 + 2.0 ** -20)])
        r = orc.sum2(x)
        _, _, A, E = orc.exact_dot_f32(x, None, r)
        assert abs(E) <= gamma(len(x)) ** 2 * A
    # sums that fit a float-float exactly come out exact
    x = np.array([1.0, 2.0 ** -30, -1.0, 2.0 ** -40, 3.0], np.float32)
    r = orc.sum2(x)
    assert Fraction(float(r[0])) + Fraction(float(r[1])) == sum(Fraction(float(v)) for v in x)


def test_dot2_reduces_to_sum2_and_twoproduct(orc):
    rng = np.random.default_rng(11)
    x = (rng.standard_normal(1000) * 2.0 ** rng.integers(-10, 10, 1000)).astype(np.float32)
    one = np.ones_like(x)
    assert np.all(orc.dot2(x, one) == orc.sum2(x))
    r = orc.dot2(x[:1], x[1:2])
    assert np.all(r == orc.mul12(np.array([[x[0], x[1]]], np.float32))[0])


def test_gemv_dA_outer_product_and_bound(orc):
    m, n = 12, 17
    gi = inputs.gemv(m, n, 1, inputs.seed_for(4, 40))
    dY, X = gi.dY.numpy(), gi.X.numpy()
    dA = orc.gemv_dA(dY, X)
    # k = 1: every element is one Mul22 (Add22 with (0, 0) returns it)
    want = orc.mul22(np.repeat(dY[0], n, axis=0), np.tile(X[0], (m, 1))).reshape(m, n, 2)
    np.testing.assert_array_equal(dA, want)
    k = 9
    gi = inputs.gemv(m, n, k, inputs.seed_for(4, 41))
    dY, X = gi.dY.numpy(), gi.X.numpy()
    dA = orc.gemv_dA(dY, X)
    for r in range(m):
        for j in range(n):
            _, _, Aabs, E = orc.exact_dot(np.ascontiguousarray(dY[:, r]), np.ascontiguousarray(X[:, j]), dA[r, j])
            assert abs(E) <= k * 2.0 ** -44 * Aabs


# --------------------------------------------------------------------------
# GEMM (many right-hand sides; Mul22 products, Add22 accumulation)
# --------------------------------------------------------------------------

def test_gemm_small_integers_exact(orc):
    """Integer matrices whose products and partial sums stay below 2^24 are
    multiplied exactly: the float-float result equals the integer product
    (numpy int64), for non-square shapes and every transpose combination."""
    rng = np.random.default_rng(11)
    m, n, kk = 5, 7, 9
    Ai = rng.integers(-300, 300, size=(m, kk))
    Bi = rng.integers(-300, 300, size=(kk, n))
    want = Ai @ Bi
    A = np.zeros((m, kk, 2), np.float32); A[..., 0] = Ai
    B = np.zeros((kk, n, 2), np.float32); B[..., 0] = Bi
    At = np.ascontiguousarray(A.transpose(1, 0, 2))
    Bt = np.ascontiguousarray(B.transpose(1, 0, 2))
    for ta, tb in ((0, 0), (1, 0), (0, 1), (1, 1)):
        C = orc.gemm(At if ta else A, Bt if tb else B, transa=bool(ta), transb=bool(tb))
        np.testing.assert_array_equal(C[..., 0].astype(np.int64), want)
        assert np.all(C[..., 1] == 0)


def test_gemm_identity_and_unit_columns(orc):
    gi = inputs.gemm(6, 11, 8, inputs.seed_for(4, 60))
    A, B = gi.A.numpy(), gi.B.numpy()
    I8 = np.zeros((8, 8, 2), np.float32); I8[np.arange(8), np.arange(8), 0] = 1.0
    I6 = np.zeros((6, 6, 2), np.float32); I6[np.arange(6), np.arange(6), 0] = 1.0
    np.testing.assert_array_equal(orc.gemm(A, I8), orc.add12(A.reshape(-1, 2)).reshape(A.shape))
    np.testing.assert_array_equal(orc.gemm(I8, B), orc.add12(B.reshape(-1, 2)).reshape(B.shape))
    np.testing.assert_array_equal(orc.gemm(I6, A), orc.add12(A.reshape(-1, 2)).reshape(A.shape))
    # a unit column of B picks out one column of A
    E = np.zeros((8, 1, 2), np.float32); E[3, 0, 0] = 1.0
    np.testing.assert_array_equal(orc.gemm(A, E)[:, 0], orc.add12(A[:, 3]))


def test_gemm_within_bound_and_transpose_identity(orc):
    """Every element within kk 2^-44 sum|a b| of the exact value (the
    superaccumulator); C^T = B^T A^T bit for bit (Mul22 with a fused Mul12
    is symmetric in its operands and the accumulation order is the same)."""
    m, n, kk = 7, 5, 133
    gi = inputs.gemm(m, n, kk, inputs.seed_for(4, 61))
    A, B = gi.A.numpy(), gi.B.numpy()
    C = orc.gemm(A, B)
    for i in range(m):
        for j in range(n):
            _, _, Aabs, Err = orc.exact_dot(A[i], np.ascontiguousarray(B[:, j]), C[i, j])
            assert abs(Err) <= kk * 2.0 ** -44 * Aabs
    Ct = orc.gemm(B, A, transa=True, transb=True)
    np.testing.assert_array_equal(Ct, np.ascontiguousarray(C.transpose(1, 0, 2)))
    # one row times one column is the float-float dot of the two
    np.testing.assert_array_equal(orc.gemm(A[2:3], B[:, 4:5])[0, 0], orc.ff_dot(A[2], np.ascontiguousarray(B[:, 4])))


def test_gemm_empty_inner_dimension(orc):
    A = np.zeros((3, 0, 2), np.float32); B = np.zeros((0, 4, 2), np.float32)
    C = orc.gemm(A, B)
    assert C.shape == (3, 4, 2) and np.all(bits(C) == 0)
