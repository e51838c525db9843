"""CPU oracle for the float-float operators -- TEST INFRASTRUCTURE ONLY.

This package binds ``liboracle.so`` (plain C, built from ``ff_oracle.c`` and
``ff_exact.c`` with ``-ffp-contract=off``) through ctypes and wraps every
entry point for numpy arrays.  Only the tests, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product path never does,
and the two share no code.

Float-float arrays are ``float32`` numpy arrays of shape ``(n, 2)`` holding
``(hi, lo)`` rows.  Packed error-free-transformation inputs are ``(n, 2)``
arrays of ``(a, b)`` rows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SOURCES = [os.path.join(HERE, f) for f in ("ff_oracle.c", "ff_exact.c")]
CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
          "-fno-unsafe-math-optimizations", "-fPIC", "-shared"]


def compile_sources(sources, out_path: str) -> str:
    """Compile the given C sources into a shared library with the oracle's
    flags."""
    tmp = out_path + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, *sources, "-lm"], check=True)
    os.replace(tmp, out_path)
    return out_path


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no contraction, no fast-math)."""
    newest = max(os.path.getmtime(s) for s in SOURCES)
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= newest):
        return LIB_PATH
    return compile_sources(SOURCES, LIB_PATH)


_lib = None


def _bind(path: str) -> ctypes.CDLL:
    L = ctypes.CDLL(path)
    _declare(L)
    return L


def swap_library(path):
    """Bind the wrappers to another build of the oracle sources (a library
    at `path`, or the default build when path is None); returns the previous
    binding's path.  Used by the tests that plant a mistake in a copy of the
    oracle and check that the pins catch it."""
    global _lib, _lib_path
    prev = _lib_path
    _lib = _bind(path) if path else None
    _lib_path = path
    return prev


_lib_path = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        _lib = _bind(LIB_PATH)
    return _lib


def _declare(L: ctypes.CDLL) -> None:
    P, S, I64, D = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_double
    sig = {
        "orc_add12": [P, P, S], "orc_split": [P, P, S],
        "orc_mul12_dekker": [P, P, S], "orc_mul12": [P, P, S],
        "orc_add22": [P, P, P, S], "orc_mul22": [P, P, P, S],
        "orc_mul22_dekker": [P, P, P, S], "orc_div22": [P, P, P, S],
        "orc_add22_accurate": [P, P, P, S], "orc_sum2": [P, S, P], "orc_dot2": [P, P, S, P],
        "exact_dot_f32": [P, P, S, P, P],
        "orc_sqrt22": [P, P, S], "orc_sum": [P, S, P],
        "orc_dot": [P, P, S, P], "orc_dot_backward": [P, P, P, P, P, S],
        "orc_axpy": [P, P, P, P, S],
        "orc_gemv": [P, I64, I64, I64, P, I64, I64, P, I64],
        "orc_gemv_t": [P, I64, I64, I64, P, I64, I64, P, I64],
        "orc_gemv_dA": [P, I64, I64, P, I64, I64, I64, P, I64],
        "orc_gemm": [ctypes.c_int, ctypes.c_int, I64, I64, I64, P, I64, P, I64, P, I64],
        "orc_fp32_add": [P, P, P, S], "orc_fp32_mul": [P, P, P, S],
        "orc_fp32_mad": [P, P, P, P, S],
        "exact_sum_f64_q": [P, S, P], "exact_count_sum2_mismatch": [P, P, S],
        "exact_count_prod_mismatch": [P, P, S], "exact_add22_bound": [P, P, P, P, S],
        "exact_relerr_ff": [ctypes.c_int, P, P, P, P, S], "exact_dot_ff": [P, P, S, P, P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = None
    L.exact_count_sum2_mismatch.restype = S
    L.exact_count_prod_mismatch.restype = S
    L.exact_sum_f64.argtypes = [P, S]
    L.exact_sum_f64.restype = D
    L.orc_canary_mul_add.argtypes = [ctypes.c_float] * 3
    L.orc_canary_mul_add.restype = ctypes.c_float


def _f32(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _pairs(a) -> np.ndarray:
    a = _f32(a)
    if a.ndim != 2 or a.shape[1] != 2:
        raise ValueError("expected an (n, 2) float32 array of pairs")
    return a


# -- error-free transformations (Section 4.1) --------------------------------

def add12(ab):
    ab = _pairs(ab); out = np.empty_like(ab)
    lib().orc_add12(_p(ab), _p(out), ab.shape[0]); return out


def split(a):
    a = _f32(a).reshape(-1); out = np.empty((a.size, 2), np.float32)
    lib().orc_split(_p(a), _p(out), a.size); return out


def mul12(ab):
    ab = _pairs(ab); out = np.empty_like(ab)
    lib().orc_mul12(_p(ab), _p(out), ab.shape[0]); return out


def mul12_dekker(ab):
    ab = _pairs(ab); out = np.empty_like(ab)
    lib().orc_mul12_dekker(_p(ab), _p(out), ab.shape[0]); return out


# -- float-float operators ---------------------------------------------------

def _binary(name, a, b):
    a = _pairs(a); b = _pairs(b)
    if a.shape != b.shape:
        raise ValueError("shape mismatch")
    out = np.empty_like(a)
    getattr(lib(), name)(_p(a), _p(b), _p(out), a.shape[0]); return out


def add22(a, b): return _binary("orc_add22", a, b)
def mul22(a, b): return _binary("orc_mul22", a, b)
def mul22_dekker(a, b): return _binary("orc_mul22_dekker", a, b)
def div22(a, b): return _binary("orc_div22", a, b)
def add22_accurate(a, b): return _binary("orc_add22_accurate", a, b)


def sum2(x):
    """Ogita-Rump-Oishi Sum2 of a binary32 vector, as an unrounded (p, s) pair."""
    x = _f32(x).reshape(-1); out = np.empty(2, np.float32)
    lib().orc_sum2(_p(x), x.size, _p(out)); return out


def dot2(x, y):
    """Ogita-Rump-Oishi Dot2 of binary32 vectors, as an unrounded (p, s) pair."""
    x = _f32(x).reshape(-1); y = _f32(y).reshape(-1); out = np.empty(2, np.float32)
    lib().orc_dot2(_p(x), _p(y), x.size, _p(out)); return out


def exact_dot_f32(x, y=None, res=None):
    """Exact reference of a binary32 dot (or sum): (S_hi, S_lo, A, E) as for
    exact_dot, with E measured for the float-float result res."""
    x = _f32(x).reshape(-1)
    yp = None
    if y is not None:
        y = _f32(y).reshape(-1); yp = _p(y)
    rp = None
    if res is not None:
        res = _f32(res).reshape(2); rp = _p(res)
    out = np.empty(4)
    lib().exact_dot_f32(_p(x), yp, x.size, rp, _p(out))
    return tuple(float(v) for v in out)


def sqrt22(a):
    a = _pairs(a); out = np.empty_like(a)
    lib().orc_sqrt22(_p(a), _p(out), a.shape[0]); return out


def ff_sum(x):
    x = _pairs(x); out = np.empty(2, np.float32)
    lib().orc_sum(_p(x), x.shape[0], _p(out)); return out


def ff_dot(x, y):
    x = _pairs(x); y = _pairs(y); out = np.empty(2, np.float32)
    lib().orc_dot(_p(x), _p(y), x.shape[0], _p(out)); return out


def dot_backward(dout, x, y):
    dout = _f32(dout).reshape(2); x = _pairs(x); y = _pairs(y)
    dx = np.empty_like(x); dy = np.empty_like(y)
    lib().orc_dot_backward(_p(dout), _p(x), _p(y), _p(dx), _p(dy), x.shape[0])
    return dx, dy


def axpy(alpha, x, y):
    alpha = _f32(alpha).reshape(2); x = _pairs(x); y = _pairs(y)
    z = np.empty_like(x)
    lib().orc_axpy(_p(alpha), _p(x), _p(y), _p(z), x.shape[0]); return z


def gemv(A, X):
    """Y = A X.  A: (m, n, 2) row-major; X: (k, n, 2) (column j of X is X[j]).
    Returns Y as (k, m, 2) (column-major m x k)."""
    A = _f32(A); X = _f32(X)
    m, n = A.shape[0], A.shape[1]
    k = X.shape[0]
    Y = np.empty((k, m, 2), np.float32)
    lib().orc_gemv(_p(A), m, n, n, _p(X), n, k, _p(Y), m); return Y


def gemv_t(A, dY):
    """dX = A^T dY.  A: (m, n, 2); dY: (k, m, 2).  Returns dX as (k, n, 2)."""
    A = _f32(A); dY = _f32(dY)
    m, n = A.shape[0], A.shape[1]
    k = dY.shape[0]
    dX = np.empty((k, n, 2), np.float32)
    lib().orc_gemv_t(_p(A), m, n, n, _p(dY), m, k, _p(dX), n); return dX


def gemm(A, B, transa=False, transb=False):
    """C = op(A) op(B), float-float, accumulated in order of the inner index.
    A: (m, kk, 2), or (kk, m, 2) when transa; B: (kk, n, 2), or (n, kk, 2)
    when transb.  Returns C as (m, n, 2)."""
    A = _f32(A); B = _f32(B)
    kk, m = (A.shape[0], A.shape[1]) if transa else (A.shape[1], A.shape[0])
    n = B.shape[0] if transb else B.shape[1]
    assert (B.shape[1] if transb else B.shape[0]) == kk
    C = np.empty((m, n, 2), np.float32)
    lib().orc_gemm(int(transa), int(transb), m, n, kk, _p(A), A.shape[1], _p(B), B.shape[1], _p(C), n)
    return C


def gemv_dA(dY, X):
    """dA = dY X^T.  dY: (k, m, 2); X: (k, n, 2).  Returns dA as (m, n, 2)."""
    dY = _f32(dY); X = _f32(X)
    k, m = dY.shape[0], dY.shape[1]
    n = X.shape[1]
    dA = np.empty((m, n, 2), np.float32)
    lib().orc_gemv_dA(_p(dY), m, m, _p(X), n, n, k, _p(dA), n); return dA


def fp32_add(a, b):
    a = _f32(a); b = _f32(b); out = np.empty_like(a)
    lib().orc_fp32_add(_p(a), _p(b), _p(out), a.size); return out


def fp32_mul(a, b):
    a = _f32(a); b = _f32(b); out = np.empty_like(a)
    lib().orc_fp32_mul(_p(a), _p(b), _p(out), a.size); return out


def fp32_mad(a, b, c):
    a = _f32(a); b = _f32(b); c = _f32(c); out = np.empty_like(a)
    lib().orc_fp32_mad(_p(a), _p(b), _p(c), _p(out), a.size); return out


def canary_mul_add(a: float, b: float, c: float) -> float:
    return lib().orc_canary_mul_add(a, b, c)


# -- exact references ----------------------------------------------------------

def exact_sum_f64(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().exact_sum_f64(_p(v), v.size)


def exact_sum_f64_q(v):
    """Exact sum of doubles rounded to binary128, as a (hi, lo) double pair."""
    v = np.ascontiguousarray(v, dtype=np.float64); out = np.empty(2)
    lib().exact_sum_f64_q(_p(v), v.size, _p(out)); return out


def count_sum2_mismatch(ab, cd) -> int:
    """How many rows have a + b != c + d exactly."""
    ab = _pairs(ab); cd = _pairs(cd)
    return lib().exact_count_sum2_mismatch(_p(ab), _p(cd), ab.shape[0])


def count_prod_mismatch(ab, xy) -> int:
    """How many rows have a * b != x + y exactly."""
    ab = _pairs(ab); xy = _pairs(xy)
    return lib().exact_count_prod_mismatch(_p(ab), _p(xy), ab.shape[0])


def add22_bound(a, b, r):
    """(|delta|, 2^-24 |al+bl|, 2^-44 |a+b|) per row, see the Add22 theorem."""
    a = _pairs(a); b = _pairs(b); r = _pairs(r)
    out = np.empty((a.shape[0], 3))
    lib().exact_add22_bound(_p(a), _p(b), _p(r), _p(out), a.shape[0]); return out


OPS = {"add": 0, "mul": 1, "div": 2, "sqrt": 3}


def relerr(op: str, a, b, r) -> np.ndarray:
    """|result - exact| / |exact| per row (binary128 reference)."""
    a = _pairs(a); r = _pairs(r)
    bp = None
    if b is not None:
        b = _pairs(b); bp = _p(b)
    out = np.empty(a.shape[0])
    lib().exact_relerr_ff(OPS[op], _p(a), bp, _p(r), _p(out), a.shape[0]); return out


def exact_dot(x, y=None, res=None):
    """Exact reference of a float-float dot (or sum when y is None).

    Returns (S_hi, S_lo, A, E): S = sum x_i y_i rounded to binary128 as a
    double pair, A = sum |x_i y_i|, E = (res_hi + res_lo) - S exactly (0 when
    res is None)."""
    x = _pairs(x)
    yp = None
    if y is not None:
        y = _pairs(y); yp = _p(y)
    rp = None
    if res is not None:
        res = _f32(res).reshape(2); rp = _p(res)
    out = np.empty(4)
    lib().exact_dot_ff(_p(x), yp, x.shape[0], rp, _p(out))
    return tuple(float(v) for v in out)
