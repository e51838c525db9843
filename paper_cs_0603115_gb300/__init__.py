"""GB300 float-float arithmetic (Da Graca & Defour, arXiv cs/0603115).

A float-float tensor is a ``torch.float32`` CUDA tensor whose last dimension
is 2: ``x[..., 0]`` is the high part and ``x[..., 1]`` the low part of the
unevaluated sum hi + lo (Section 4 of the paper).  Vectors are ``(n, 2)``.
Every function here marshals its arguments and calls one entry point of the
C ABI in ``libff.so`` (include/ff.h) on the current CUDA stream; all
arithmetic runs in the library's CUDA kernels.  Nothing falls back to the CPU:
a missing library or a non-CUDA tensor raises.

Elementwise:  add12, mul12 (packed (a, b) pairs), add, add_accurate, mul, div,
              sqrt, axpy
Reductions:   sum, dot (device-resident float-float result), sum2, dot2
              (binary32 inputs), dot_backward
GEMV, GEMM:   gemv (Y = A X), gemv_t (dX = A^T dY), gemv_dA (dA = dY X^T),
              gemm (C = op(A) op(B))
Autograd:     FFDot, FFGemv, FFGemm and ffdot, ffgemv, ffgemm (hand-written
              adjoint kernels)
Baselines:    f64_add/mul/div/sqrt/dot/gemv, f32_add/mul/mad, fma_peak
Submodules:   batch (many instances in one persistent launch, CUDA graphs,
              autotuner), dist (sharded reductions over processes), inputs
              (the seeded input recipe)
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import FFError, ff2

__all__ = [
    "add12", "mul12", "add", "add_accurate", "sum2", "dot2", "mul", "div", "sqrt", "axpy", "sum", "dot", "dot_backward",
    "gemv", "gemv_t", "gemv_dA", "gemm", "FFDot", "FFGemv", "FFGemm", "ffdot", "ffgemv", "ffgemm", "FFError",
    "workspace", "clear_workspaces",
    "f64_add", "f64_mul", "f64_div", "f64_sqrt", "f64_dot", "f64_gemv", "f32_add", "f32_mul",
    "f32_mad", "fma_peak", "load",
]


def load():
    """Load libff.so (raises if it is not built)."""
    return _lib.load()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _check_device(t: torch.Tensor, name: str) -> None:
    """Kernels launch on the current device with the current stream: every
    tensor must live there (a tensor of another GPU would be read through a
    pointer that device cannot use)."""
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")
    cur = torch.cuda.current_device()
    if t.device.index != cur:
        raise ValueError(f"{name}: tensor on {t.device} but the current device is cuda:{cur} "
                         f"(use torch.cuda.device({t.device.index}))")


def _check_ff(t: torch.Tensor, name: str) -> None:
    _check_device(t, name)
    if t.dtype != torch.float32 or t.dim() < 1 or t.shape[-1] != 2:
        raise ValueError(f"{name}: expected float32 with a last dimension of 2, got {t.dtype} {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")


def _check_out(t: torch.Tensor, name: str, shape, dtype=torch.float32) -> None:
    """A caller-supplied output must have exactly the result's shape and
    dtype, be contiguous and live on the current device: the kernels write
    through a plain pointer and cannot see its extent."""
    _check_device(t, name)
    if t.dtype != dtype or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: output must be a contiguous {dtype} tensor of shape {tuple(shape)}, "
                         f"got {t.dtype} {tuple(t.shape)}{'' if t.is_contiguous() else ' (not contiguous)'}")


def _nvals(t: torch.Tensor) -> int:
    return t.numel() // 2


# ---------------------------------------------------------------------------
# workspace (caller-owned device scratch, cached per device and stream)
# ---------------------------------------------------------------------------
_ws_cache: dict = {}


def workspace(nbytes: int, device=None, key: str = "reduce") -> torch.Tensor:
    """A cached uint8 device buffer of at least ``nbytes`` (16-byte aligned)
    for calls on the current stream.

    Each (device, stream, key) has its own buffer, allocated while that
    stream is current, so calls on one stream reuse it in stream order and
    calls on different streams never share one.  Buffers start zeroed (a
    reduction workspace's arrival ticket must be zero before its first use;
    each reduction leaves it zero).  A GEMV-adjoint workspace can be large
    (row blocks x n x k values); ``clear_workspaces()`` releases every cached
    buffer."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    k = (dev.index, torch.cuda.current_stream(dev).cuda_stream, key)
    buf = _ws_cache.get(k)
    if buf is None or buf.numel() < nbytes:
        buf = torch.zeros(max(int(nbytes), 256), dtype=torch.uint8, device=dev)
        _ws_cache[k] = buf
    return buf


def clear_workspaces() -> None:
    """Drop every cached workspace (the memory returns to PyTorch's caching
    allocator once the work already enqueued on their streams has run)."""
    _ws_cache.clear()


# ---------------------------------------------------------------------------
# elementwise
# ---------------------------------------------------------------------------
def _unary(name, x, out):
    _check_ff(x, name)
    if out is None:
        out = torch.empty_like(x)
    _check_ff(out, name)
    if out.shape != x.shape:
        raise ValueError(f"{name}: output shape mismatch")
    _lib.call(name, _ptr(x), _ptr(out), _nvals(x), _stream())
    return out


def _binary(name, a, b, out):
    _check_ff(a, name)
    _check_ff(b, name)
    if a.shape != b.shape:
        raise ValueError(f"{name}: shape mismatch {tuple(a.shape)} vs {tuple(b.shape)}")
    if out is None:
        out = torch.empty_like(a)
    _check_ff(out, name)
    if out.shape != a.shape:
        raise ValueError(f"{name}: output shape mismatch")
    _lib.call(name, _ptr(a), _ptr(b), _ptr(out), _nvals(a), _stream())
    return out


def add12(ab, out=None):
    """Add12 on packed binary32 pairs: (s, e), s = RN(a + b), s + e = a + b."""
    return _unary("ff_add12", ab, out)


def mul12(ab, out=None):
    """Mul12 on packed binary32 pairs: (p, e), p = RN(a b), p + e = a b."""
    return _unary("ff_mul12", ab, out)


def add(a, b, out=None):
    """Add22: float-float a + b."""
    return _binary("ff_add", a, b, out)


def add_accurate(a, b, out=None):
    """Accurate float-float a + b (Joldes-Muller-Popescu), relative error
    <= 3 2^-48 / (1 - 2^-22) even under cancellation."""
    return _binary("ff_add_accurate", a, b, out)


def mul(a, b, out=None):
    """Mul22: float-float a * b."""
    return _binary("ff_mul", a, b, out)


def div(a, b, out=None):
    """Div22: float-float a / b."""
    return _binary("ff_div", a, b, out)


def sqrt(a, out=None):
    """Sqrt22: float-float sqrt(a)."""
    return _unary("ff_sqrt", a, out)


def axpy(alpha, x, y, out=None):
    """z = Add22(Mul22(alpha, x), y); alpha is a (hi, lo) pair of floats."""
    _check_ff(x, "ff_axpy")
    _check_ff(y, "ff_axpy")
    if x.shape != y.shape:
        raise ValueError("ff_axpy: shape mismatch")
    if out is None:
        out = torch.empty_like(x)
    _check_out(out, "ff_axpy", x.shape)
    hi, lo = (float(alpha[0]), float(alpha[1]))
    _lib.call("ff_axpy", ff2(hi, lo), _ptr(x), _ptr(y), _ptr(out), _nvals(x), _stream())
    return out


# ---------------------------------------------------------------------------
# reductions
# ---------------------------------------------------------------------------
def _reduce_ws(n: int, device) -> torch.Tensor:
    return workspace(_lib.load().ff_reduce_workspace_bytes(n), device)


def sum(x, out=None):  # noqa: A001  (mirrors the C name ff_sum)
    """Float-float sum of an (n, 2) vector; returns a (2,) device tensor."""
    _check_ff(x, "ff_sum")
    if out is None:
        out = torch.empty(2, dtype=torch.float32, device=x.device)
    _check_out(out, "ff_sum", (2,))
    n = _nvals(x)
    ws = _reduce_ws(n, x.device)
    _lib.call("ff_sum", _ptr(x), n, _ptr(out), _ptr(ws), ws.numel(), _stream())
    return out


def dot(x, y, out=None):
    """Float-float dot product sum_i Mul22(x_i, y_i); returns (2,) on device."""
    _check_ff(x, "ff_dot")
    _check_ff(y, "ff_dot")
    if x.shape != y.shape:
        raise ValueError("ff_dot: shape mismatch")
    if out is None:
        out = torch.empty(2, dtype=torch.float32, device=x.device)
    _check_out(out, "ff_dot", (2,))
    n = _nvals(x)
    ws = _reduce_ws(n, x.device)
    _lib.call("ff_dot", _ptr(x), _ptr(y), n, _ptr(out), _ptr(ws), ws.numel(), _stream())
    return out


def _f32_vec(t, name):
    _check_device(t, name)
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous float32 CUDA tensor")


def sum2(x, out=None):
    """Compensated Sum2 of a binary32 vector; returns the float-float (2,)
    result on the device."""
    _f32_vec(x, "ff_sum2")
    if out is None:
        out = torch.empty(2, dtype=torch.float32, device=x.device)
    _check_out(out, "ff_sum2", (2,))
    ws = _reduce_ws(x.numel(), x.device)
    _lib.call("ff_sum2", _ptr(x), x.numel(), _ptr(out), _ptr(ws), ws.numel(), _stream())
    return out


def dot2(x, y, out=None):
    """Compensated Dot2 of binary32 vectors; returns the float-float (2,)
    result on the device."""
    _f32_vec(x, "ff_dot2")
    _f32_vec(y, "ff_dot2")
    if x.numel() != y.numel():
        raise ValueError("ff_dot2: size mismatch")
    if out is None:
        out = torch.empty(2, dtype=torch.float32, device=x.device)
    _check_out(out, "ff_dot2", (2,))
    ws = _reduce_ws(x.numel(), x.device)
    _lib.call("ff_dot2", _ptr(x), _ptr(y), x.numel(), _ptr(out), _ptr(ws), ws.numel(), _stream())
    return out


def dot_backward(dout, x, y, dx=None, dy=None):
    """dx = Mul22(dout, y), dy = Mul22(dout, x); dout is a (2,) device tensor."""
    _check_ff(dout, "ff_dot_backward")
    _check_ff(x, "ff_dot_backward")
    _check_ff(y, "ff_dot_backward")
    if dout.numel() != 2 or x.shape != y.shape:
        raise ValueError("ff_dot_backward: expected dout of 2 values and x, y of one shape")
    if dx is None:
        dx = torch.empty_like(x)
    if dy is None:
        dy = torch.empty_like(y)
    _check_out(dx, "ff_dot_backward", x.shape)
    _check_out(dy, "ff_dot_backward", y.shape)
    _lib.call("ff_dot_backward", _ptr(dout), _ptr(x), _ptr(y), _ptr(dx), _ptr(dy), _nvals(x), _stream())
    return dx, dy


# ---------------------------------------------------------------------------
# GEMV
# ---------------------------------------------------------------------------
def gemv(A, X, out=None):
    """Y = A X.  A: (m, n, 2) row-major; X: (k, n, 2), i.e. n x k column-major
    (X[c] is right-hand side c).  Returns Y as (k, m, 2)."""
    _check_ff(A, "ff_gemv")
    _check_ff(X, "ff_gemv")
    if A.dim() != 3 or X.dim() != 3 or X.shape[1] != A.shape[1]:
        raise ValueError("ff_gemv: expected A (m, n, 2) and X (k, n, 2)")
    m, n = A.shape[0], A.shape[1]
    k = X.shape[0]
    if out is None:
        out = torch.empty((k, m, 2), dtype=torch.float32, device=A.device)
    _check_out(out, "ff_gemv", (k, m, 2))
    _lib.call("ff_gemv", _ptr(A), m, n, n, _ptr(X), n, k, _ptr(out), m, _stream())
    return out


def gemv_t(A, dY, out=None):
    """dX = A^T dY.  A: (m, n, 2); dY: (k, m, 2).  Returns dX as (k, n, 2)."""
    _check_ff(A, "ff_gemv_t")
    _check_ff(dY, "ff_gemv_t")
    if A.dim() != 3 or dY.dim() != 3 or dY.shape[1] != A.shape[0]:
        raise ValueError("ff_gemv_t: expected A (m, n, 2) and dY (k, m, 2)")
    m, n = A.shape[0], A.shape[1]
    k = dY.shape[0]
    if out is None:
        out = torch.empty((k, n, 2), dtype=torch.float32, device=A.device)
    _check_out(out, "ff_gemv_t", (k, n, 2))
    nbytes = _lib.load().ff_gemv_t_workspace_bytes(m, n, k)
    ws = workspace(nbytes, A.device, key="gemv_t")
    _lib.call("ff_gemv_t", _ptr(A), m, n, n, _ptr(dY), m, k, _ptr(out), n, _ptr(ws), ws.numel(), _stream())
    return out


def gemv_dA(dY, X, out=None):
    """dA = dY X^T (the weight gradient of Y = A X).  dY: (k, m, 2); X: (k, n, 2).
    Returns dA as (m, n, 2) row-major."""
    _check_ff(dY, "ff_gemv_dA")
    _check_ff(X, "ff_gemv_dA")
    if dY.dim() != 3 or X.dim() != 3 or dY.shape[0] != X.shape[0]:
        raise ValueError("ff_gemv_dA: expected dY (k, m, 2) and X (k, n, 2)")
    k, m = dY.shape[0], dY.shape[1]
    n = X.shape[1]
    if out is None:
        out = torch.empty((m, n, 2), dtype=torch.float32, device=dY.device)
    _check_out(out, "ff_gemv_dA", (m, n, 2))
    _lib.call("ff_gemv_dA", _ptr(dY), m, m, _ptr(X), n, n, k, _ptr(out), n, _stream())
    return out


def gemm(A, B, transa=False, transb=False, out=None):
    """C = op(A) op(B), row-major float-float matrices.  A: (m, k, 2), or
    (k, m, 2) when transa; B: (k, n, 2), or (n, k, 2) when transb.  Returns C
    as (m, n, 2)."""
    _check_ff(A, "ff_gemm")
    _check_ff(B, "ff_gemm")
    if A.dim() != 3 or B.dim() != 3:
        raise ValueError("ff_gemm: expected A and B of shape (rows, cols, 2)")
    k, m = (A.shape[0], A.shape[1]) if transa else (A.shape[1], A.shape[0])
    kb, n = (B.shape[1], B.shape[0]) if transb else (B.shape[0], B.shape[1])
    if kb != k:
        raise ValueError(f"ff_gemm: inner dimensions differ ({k} and {kb})")
    if out is None:
        out = torch.empty((m, n, 2), dtype=torch.float32, device=A.device)
    _check_out(out, "ff_gemm", (m, n, 2))
    _lib.call("ff_gemm", int(bool(transa)), int(bool(transb)), m, n, k, _ptr(A), max(A.shape[1], 1), _ptr(B),
              max(B.shape[1], 1), _ptr(out), max(n, 1), _stream())
    return out


# ---------------------------------------------------------------------------
# autograd: hand-written adjoints
# ---------------------------------------------------------------------------
class FFDot(torch.autograd.Function):
    """d = dot(x, y) with the adjoint kernel ff_dot_backward.  The gradient of
    a float-float tensor is a float-float tensor holding dL/d(hi + lo).  The
    backward reuses the inputs themselves (saved by reference); nothing else
    is stored."""

    @staticmethod
    def forward(ctx, x, y):
        ctx.save_for_backward(x, y)
        return dot(x, y)

    @staticmethod
    def backward(ctx, dout):
        x, y = ctx.saved_tensors
        dout = dout.contiguous()
        dx, dy = dot_backward(dout, x, y)
        return (dx if ctx.needs_input_grad[0] else None, dy if ctx.needs_input_grad[1] else None)


class FFGemv(torch.autograd.Function):
    """Y = A X with the adjoints dX = A^T dY (ff_gemv_t) and, when A needs a
    gradient, dA = dY X^T (ff_gemv_dA)."""

    @staticmethod
    def forward(ctx, A, X):
        ctx.save_for_backward(A, X)
        return gemv(A, X)

    @staticmethod
    def backward(ctx, dY):
        A, X = ctx.saved_tensors
        dY = dY.contiguous()
        dA = gemv_dA(dY, X) if ctx.needs_input_grad[0] else None
        dX = gemv_t(A, dY) if ctx.needs_input_grad[1] else None
        return dA, dX


class FFGemm(torch.autograd.Function):
    """C = A B with the adjoints dA = dC B^T and dB = A^T dC, both ff_gemm
    launches on the stored operands (no transposed copies)."""

    @staticmethod
    def forward(ctx, A, B):
        ctx.save_for_backward(A, B)
        return gemm(A, B)

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dC = dC.contiguous()
        dA = gemm(dC, B, transb=True) if ctx.needs_input_grad[0] else None
        dB = gemm(A, dC, transa=True) if ctx.needs_input_grad[1] else None
        return dA, dB


def ffdot(x, y):
    return FFDot.apply(x, y)


def ffgemv(A, X):
    return FFGemv.apply(A, X)


def ffgemm(A, B):
    return FFGemm.apply(A, B)


# ---------------------------------------------------------------------------
# native baselines
# ---------------------------------------------------------------------------
def _f64_check(t, name):
    _check_device(t, name)
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous float64 CUDA tensor")


def _f64_binary(name, a, b, out):
    _f64_check(a, name)
    _f64_check(b, name)
    if a.shape != b.shape:
        raise ValueError(f"{name}: shape mismatch")
    out = torch.empty_like(a) if out is None else out
    _check_out(out, name, a.shape, torch.float64)
    _lib.call(name, _ptr(a), _ptr(b), _ptr(out), a.numel(), _stream())
    return out


def f64_add(a, b, out=None): return _f64_binary("ff_f64_add", a, b, out)
def f64_mul(a, b, out=None): return _f64_binary("ff_f64_mul", a, b, out)
def f64_div(a, b, out=None): return _f64_binary("ff_f64_div", a, b, out)


def f64_sqrt(a, out=None):
    _f64_check(a, "ff_f64_sqrt")
    out = torch.empty_like(a) if out is None else out
    _check_out(out, "ff_f64_sqrt", a.shape, torch.float64)
    _lib.call("ff_f64_sqrt", _ptr(a), _ptr(out), a.numel(), _stream())
    return out


def f64_dot(x, y, out=None):
    _f64_check(x, "ff_f64_dot")
    _f64_check(y, "ff_f64_dot")
    if x.shape != y.shape:
        raise ValueError("ff_f64_dot: shape mismatch")
    out = torch.empty(1, dtype=torch.float64, device=x.device) if out is None else out
    _check_out(out, "ff_f64_dot", (1,), torch.float64)
    ws = _reduce_ws(x.numel(), x.device)
    _lib.call("ff_f64_dot", _ptr(x), _ptr(y), x.numel(), _ptr(out), _ptr(ws), ws.numel(), _stream())
    return out


def f64_gemv(A, X, out=None):
    """Binary64 Y = A X; A (m, n), X (k, n); returns (k, m)."""
    _f64_check(A, "ff_f64_gemv")
    _f64_check(X, "ff_f64_gemv")
    if A.dim() != 2 or X.dim() != 2 or X.shape[1] != A.shape[1]:
        raise ValueError("ff_f64_gemv: expected A (m, n) and X (k, n)")
    m, n = A.shape
    k = X.shape[0]
    out = torch.empty((k, m), dtype=torch.float64, device=A.device) if out is None else out
    _check_out(out, "ff_f64_gemv", (k, m), torch.float64)
    _lib.call("ff_f64_gemv", _ptr(A), m, n, n, _ptr(X), n, k, _ptr(out), m, _stream())
    return out


def _f32_check(t, name):
    _check_device(t, name)
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous float32 CUDA tensor")


def f32_add(a, b, out=None):
    _f32_check(a, "ff_f32_add"); _f32_check(b, "ff_f32_add")
    if a.shape != b.shape:
        raise ValueError("ff_f32_add: shape mismatch")
    out = torch.empty_like(a) if out is None else out
    _check_out(out, "ff_f32_add", a.shape)
    _lib.call("ff_f32_add", _ptr(a), _ptr(b), _ptr(out), a.numel(), _stream())
    return out


def f32_mul(a, b, out=None):
    _f32_check(a, "ff_f32_mul"); _f32_check(b, "ff_f32_mul")
    if a.shape != b.shape:
        raise ValueError("ff_f32_mul: shape mismatch")
    out = torch.empty_like(a) if out is None else out
    _check_out(out, "ff_f32_mul", a.shape)
    _lib.call("ff_f32_mul", _ptr(a), _ptr(b), _ptr(out), a.numel(), _stream())
    return out


def f32_mad(a, b, c, out=None):
    for t in (a, b, c):
        _f32_check(t, "ff_f32_mad")
    if a.shape != b.shape or a.shape != c.shape:
        raise ValueError("ff_f32_mad: shape mismatch")
    out = torch.empty_like(a) if out is None else out
    _check_out(out, "ff_f32_mad", a.shape)
    _lib.call("ff_f32_mad", _ptr(a), _ptr(b), _ptr(c), _ptr(out), a.numel(), _stream())
    return out


def fma_peak(f64: bool, iters: int, blocks: int, threads: int = 256, device=None, out=None):
    """Launch the FMA throughput probe (16 * iters * blocks * threads flops);
    returns the per-thread sums (each 28 + 8 * iters)."""
    dtype = torch.float64 if f64 else torch.float32
    if out is None:
        out = torch.empty(blocks * threads, dtype=dtype, device=device or "cuda")
    _check_out(out, "ff_fma_peak", (blocks * threads,), dtype)
    _lib.call("ff_fma_peak", int(bool(f64)), iters, blocks, threads, _ptr(out), _stream())
    return out
