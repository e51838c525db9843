"""Property-based pins of the oracle (hypothesis searches for counterexamples
across the binary32 range; skipped where hypothesis is not installed).
Exact references are Python fractions, independent of the oracle."""
from fractions import Fraction

import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, assume  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

f32 = np.float32
F = Fraction
SETTINGS = settings(max_examples=1500, deadline=None, derandomize=True)
finite32 = st.floats(width=32, allow_nan=False, allow_infinity=False)


def ffval(hi, lo):
    return F(float(hi)) + F(float(lo))


def ffpair(draw_hi, draw_lo_scale):
    """A normalised float-float value: lo is a binary32 value at most half an
    ulp of hi."""
    hi = f32(draw_hi)
    ulp = float(np.spacing(np.abs(hi))) if hi != 0 else 0.0
    lo = f32(draw_lo_scale * ulp / 2)
    if abs(float(lo)) > ulp / 2:
        lo = f32(0.0)
    return hi, lo


@SETTINGS
@given(finite32, finite32)
def test_add12_is_exact_everywhere(orc, a, b):
    a, b = f32(a), f32(b)
    with np.errstate(over="ignore"):
        assume(np.isfinite(a + b))
    s, e = orc.add12(np.array([[a, b]], np.float32))[0]
    assert s == f32(a + b)                              # s is the rounded sum
    assert F(float(s)) + F(float(e)) == F(float(a)) + F(float(b))   # and e its exact error


@SETTINGS
@given(st.floats(min_value=2.0 ** -50, max_value=2.0 ** 50, width=32), st.floats(min_value=2.0 ** -50, max_value=2.0 ** 50, width=32),
       st.booleans(), st.booleans())
def test_mul12_is_exact_in_its_domain(orc, a, b, sa, sb):
    a, b = f32(-a if sa else a), f32(-b if sb else b)
    for fn in (orc.mul12, orc.mul12_dekker):
        p, e = fn(np.array([[a, b]], np.float32))[0]
        assert F(float(p)) + F(float(e)) == F(float(a)) * F(float(b))


mag = st.floats(min_value=2.0 ** -30, max_value=2.0 ** 30, width=32)
lo_scale = st.floats(min_value=-1.0, max_value=1.0)


@SETTINGS
@given(mag, lo_scale, mag, lo_scale, st.booleans(), st.booleans())
def test_add22_meets_its_bound(orc, ah, al, bh, bl, sa, sb):
    a = ffpair(-ah if sa else ah, al)
    b = ffpair(-bh if sb else bh, bl)
    r = orc.add22(np.array([a], np.float32), np.array([b], np.float32))[0]
    exact = ffval(*a) + ffval(*b)
    err = abs(ffval(*r) - exact)
    bound = max(F(1, 2 ** 24) * abs(F(float(a[1])) + F(float(b[1]))), F(1, 2 ** 44) * abs(exact))
    assert err <= bound


@SETTINGS
@given(mag, lo_scale, mag, lo_scale, st.booleans(), st.booleans())
def test_mul22_div22_meet_2m44(orc, ah, al, bh, bl, sa, sb):
    a = ffpair(-ah if sa else ah, al)
    b = ffpair(-bh if sb else bh, bl)
    A, B = np.array([a], np.float32), np.array([b], np.float32)
    exact = ffval(*a) * ffval(*b)
    assert abs(ffval(*orc.mul22(A, B)[0]) - exact) <= F(1, 2 ** 44) * abs(exact)
    q = ffval(*a) / ffval(*b)
    assert abs(ffval(*orc.div22(A, B)[0]) - q) <= F(1, 2 ** 44) * abs(q)


@SETTINGS
@given(mag, lo_scale)
def test_sqrt22_meets_2m44(orc, ah, al):
    a = ffpair(ah, al)
    r = orc.sqrt22(np.array([a], np.float32))[0]
    # |r^2 - a| <= 2 * 2^-44 * a  is implied by a relative error <= 2^-44 of r
    v = ffval(*a)
    rv = ffval(*r)
    assert abs(rv * rv - v) <= F(2, 2 ** 44) * v * (1 + F(1, 2 ** 43))
