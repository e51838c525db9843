"""ctypes binding of libff.so (the C ABI declared in include/ff.h).

Marshalling only: every entry point here forwards plain pointers, sizes and a
stream handle to the library; all arithmetic runs in the library's CUDA
kernels.  There is no fallback: if libff.so is missing or does not load, the
first call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
# FF_LIBRARY may name another build of the same sources (e.g. a variant
# compiled with different flags); by default the in-tree libff.so
LIB_PATH = os.environ.get("FF_LIBRARY") or os.path.join(HERE, "libff.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ff.h")


class ff2(ctypes.Structure):
    _fields_ = [("hi", ctypes.c_float), ("lo", ctypes.c_float)]


class ff_batch_instance(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("n", ctypes.c_int64),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("out2", ctypes.c_void_p), ("dout", ctypes.c_void_p), ("alpha", ff2),
                ("m", ctypes.c_int64), ("lda", ctypes.c_int64)]


class ff_tune(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("pairs_per_thread", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("unroll", ctypes.c_int32)]


P = ctypes.c_void_p
SZ = ctypes.c_size_t
I64 = ctypes.c_int64
ST = ctypes.c_int

SIGNATURES = {
    "ff_add12": (ST, [P, P, SZ, P]),
    "ff_mul12": (ST, [P, P, SZ, P]),
    "ff_add": (ST, [P, P, P, SZ, P]),
    "ff_mul": (ST, [P, P, P, SZ, P]),
    "ff_add_accurate": (ST, [P, P, P, SZ, P]),
    "ff_sum2": (ST, [P, SZ, P, P, SZ, P]),
    "ff_dot2": (ST, [P, P, SZ, P, P, SZ, P]),
    "ff_reduce2_launch_shape": (ST, [P, P, SZ, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]),
    "ff_div": (ST, [P, P, P, SZ, P]),
    "ff_sqrt": (ST, [P, P, SZ, P]),
    "ff_axpy": (ST, [ff2, P, P, P, SZ, P]),
    "ff_reduce_workspace_bytes": (SZ, [SZ]),
    "ff_sum": (ST, [P, SZ, P, P, SZ, P]),
    "ff_dot": (ST, [P, P, SZ, P, P, SZ, P]),
    "ff_dot_backward": (ST, [P, P, P, P, P, SZ, P]),
    "ff_dot_noalloc": (ST, [P, P, SZ, P, P]),
    "ff_reduce_launch_shape": (ST, [P, P, SZ, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]),
    "ff_gemv": (ST, [P, I64, I64, I64, P, I64, I64, P, I64, P]),
    "ff_gemv_t_workspace_bytes": (SZ, [I64, I64, I64]),
    "ff_gemv_t": (ST, [P, I64, I64, I64, P, I64, I64, P, I64, P, SZ, P]),
    "ff_gemv_t_launch_shape": (ST, [P, I64, I64, I64, I64, P, P]),
    "ff_gemv_dA": (ST, [P, I64, I64, P, I64, I64, I64, P, I64, P]),
    "ff_fma_peak": (ST, [ctypes.c_int, I64, ctypes.c_int, ctypes.c_int, P, P]),
    "ff_gemm": (ST, [ctypes.c_int, ctypes.c_int, I64, I64, I64, P, I64, P, I64, P, I64, P]),
    "ff_f64_add": (ST, [P, P, P, SZ, P]),
    "ff_f64_mul": (ST, [P, P, P, SZ, P]),
    "ff_f64_div": (ST, [P, P, P, SZ, P]),
    "ff_f64_sqrt": (ST, [P, P, SZ, P]),
    "ff_f64_dot": (ST, [P, P, SZ, P, P, SZ, P]),
    "ff_f64_gemv": (ST, [P, I64, I64, I64, P, I64, I64, P, I64, P]),
    "ff_f32_add": (ST, [P, P, P, SZ, P]),
    "ff_f32_mul": (ST, [P, P, P, SZ, P]),
    "ff_f32_mad": (ST, [P, P, P, P, SZ, P]),
    "ff_batch_plan_create": (ST, [P, ctypes.c_int, P, ctypes.POINTER(ctypes.c_void_p)]),
    "ff_batch_workspace_bytes": (SZ, [P]),
    "ff_batch_plan_info": (ST, [P, P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint)]),
    "ff_batch_run": (ST, [P, P, SZ, P]),
    "ff_batch_plan_destroy": (None, [P]),
    "ff_batch_graph_create": (ST, [P, P, SZ, ctypes.POINTER(ctypes.c_void_p)]),
    "ff_batch_graph_launch": (ST, [P, P]),
    "ff_batch_graph_destroy": (None, [P]),
    "ff_batch_tune_candidates": (ctypes.c_int, [P, ctypes.c_int]),
    "ff_batch_autotune_workspace_bytes": (SZ, [P, ctypes.c_int]),
    "ff_batch_autotune": (ST, [P, ctypes.c_int, P, SZ, P, ctypes.c_int, P, ctypes.POINTER(ctypes.c_float)]),
    "ff_status_string": (ctypes.c_char_p, [ST]),
    "ff_last_cuda_error": (ST, [ctypes.POINTER(ctypes.c_int)]),
    "ff_build_id": (ctypes.c_char_p, []),
}

_lib = None


class FFError(RuntimeError):
    def __init__(self, fn: str, status: int, cuda_err: int = 0):
        name = _lib.ff_status_string(status).decode() if _lib else str(status)
        msg = f"{fn} failed: {name}"
        if cuda_err:
            msg += f" (CUDA error {cuda_err})"
        super().__init__(msg)
        self.status = status
        self.cuda_err = cuda_err


def declared_symbols() -> list[str]:
    """Every function name declared in include/ff.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ff_[A-Za-z0-9_]+)\s*\(", text)))


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def call(name: str, *args) -> None:
    """Call an ff_* entry point and raise FFError on a non-zero status."""
    L = load()
    st = getattr(L, name)(*args)
    if st != 0:
        err = ctypes.c_int(0)
        L.ff_last_cuda_error(ctypes.byref(err))
        raise FFError(name, st, err.value if st == 3 else 0)
