"""The C ABI library builds, loads and exports every symbol include/ff.h
declares, and its host-side argument checks return status codes without
touching a GPU.  No test here launches a kernel."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_cs_0603115_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    from paper_cs_0603115_gb300 import _lib
    declared = _lib.declared_symbols()
    assert len(declared) >= 25
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    # the binding declares a signature for every entry point of the header
    assert sorted(_lib.SIGNATURES) == declared


def test_build_id_and_status_strings(lib):
    assert len(lib.ff_build_id()) > 0
    assert lib.ff_status_string(0) == b"FF_OK"
    assert lib.ff_status_string(2) == b"FF_ERR_WORKSPACE"
    err = ctypes.c_int(-1)
    assert lib.ff_last_cuda_error(ctypes.byref(err)) == 0
    assert lib.ff_last_cuda_error(None) == 1


def test_invalid_arguments_rejected_on_host(lib):
    INVALID = 1
    good = 1 << 20          # never dereferenced: every call below fails its checks
    mis = good + 4          # not 8-byte aligned
    assert lib.ff_add(None, good, good, 10, None) == INVALID
    assert lib.ff_add(good, good, None, 10, None) == INVALID
    assert lib.ff_add(mis, good, good, 10, None) == INVALID
    assert lib.ff_mul12(good, None, 5, None) == INVALID
    assert lib.ff_sqrt(None, good, 1, None) == INVALID
    assert lib.ff_dot(None, good, 3, good, good, 4096, None) == INVALID
    assert lib.ff_sum(good, 3, None, good, 4096, None) == INVALID
    assert lib.ff_dot_backward(good, None, good, good, good, 3, None) == INVALID
    assert lib.ff_gemv(good, 4, 4, 3, good, 4, 1, good, 4, None) == INVALID   # lda < n
    assert lib.ff_gemv(good, 4, 4, 4, good, 4, 0, good, 4, None) == INVALID   # k < 1
    assert lib.ff_gemv(good, 4, 4, 4, good, 4, 65, good, 4, None) == INVALID  # k > 64
    assert lib.ff_gemv(good, -1, 4, 4, good, 4, 1, good, 4, None) == INVALID
    assert lib.ff_gemv_t(good, 4, 4, 4, good, 3, 1, good, 4, good, 1 << 20, None) == INVALID
    assert lib.ff_f64_add(good, mis, good, 3, None) == INVALID
    assert lib.ff_gemm(2, 0, 4, 4, 4, good, 4, good, 4, good, 4, None) == INVALID   # transa not 0/1
    assert lib.ff_gemm(0, 0, 4, 4, 5, good, 4, good, 4, good, 4, None) == INVALID   # lda < k
    assert lib.ff_gemm(1, 0, 6, 4, 5, good, 5, good, 4, good, 4, None) == INVALID   # transposed: lda < m
    assert lib.ff_gemm(0, 1, 4, 6, 5, good, 5, good, 4, good, 6, None) == INVALID   # transposed: ldb < k
    assert lib.ff_gemm(0, 0, 4, 6, 5, good, 5, good, 6, good, 5, None) == INVALID   # ldc < n
    assert lib.ff_gemm(0, 0, -1, 4, 4, good, 4, good, 4, good, 4, None) == INVALID
    assert lib.ff_gemm(0, 0, 4, 4, 4, mis, 4, good, 4, good, 4, None) == INVALID
    assert lib.ff_fma_peak(2, 10, 1, 64, good, None) == INVALID
    assert lib.ff_fma_peak(0, 10, 1, 48, good, None) == INVALID     # threads not a multiple of 32
    assert lib.ff_fma_peak(0, -1, 1, 64, good, None) == INVALID
    assert lib.ff_fma_peak(1, 10, 0, 64, good, None) == INVALID
    assert lib.ff_fma_peak(1, 10, 1, 64, None, None) == INVALID


def test_zero_length_is_a_host_noop(lib):
    # n == 0: nothing to launch, no pointer needed
    assert lib.ff_add(None, None, None, 0, None) == 0
    assert lib.ff_add12(None, None, 0, None) == 0
    assert lib.ff_f32_add(None, None, None, 0, None) == 0
    assert lib.ff_gemm(0, 0, 0, 5, 3, None, 3, None, 5, None, 5, None) == 0
    assert lib.ff_gemm(0, 0, 5, 0, 3, None, 3, None, 1, None, 1, None) == 0


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_cs_0603115_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "orc_" not in text, f
    # the C sources of the oracle and the CUDA library share no file
    csrc = set(os.listdir(os.path.join(pkg, "csrc")))
    assert not (csrc & set(os.listdir(os.path.join(ROOT, "oracle"))))


def _header_prototypes():
    """(name -> (return type, [parameter types])) of every FF_API function in
    include/ff.h, comments removed, parameter names dropped."""
    from paper_cs_0603115_gb300 import _lib
    text = open(_lib.HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = {}
    for ret, name, params in re.findall(r"FF_API\s+([\w\s\*]+?)\s*\b(ff_\w+)\s*\(([^)]*)\)\s*;", text):
        types = []
        for p in params.split(","):
            p = " ".join(p.split())
            if not p or p == "void":
                continue
            types.append(re.sub(r"\s*\b\w+$", "", p) if not p.endswith("*") else p)
        protos[name] = (" ".join(ret.split()), types)
    return protos


def _ctypes_kind(t):
    """A coarse class of a C parameter or return type for the comparison."""
    t = t.replace("const ", "").strip()
    if t.endswith("*") or t in ("cudaStream_t", "ff_batch_plan", "ff_batch_graph"):
        return "pointer"
    return {"size_t": "size", "int64_t": "int64", "int": "int", "ff_status": "int", "ff2": "ff2",
            "void": "void"}[t]


def test_binding_signatures_match_the_header():
    """Every entry point's ctypes signature has the header's parameter count
    and, parameter by parameter, the same kind of type (pointer, size_t,
    int64_t, int, ff2 by value), and the same kind of return value: a
    mismatched width would pass wrong values through the ABI silently."""
    from paper_cs_0603115_gb300 import _lib
    protos = _header_prototypes()
    assert set(protos) == set(_lib.SIGNATURES), set(protos) ^ set(_lib.SIGNATURES)
    py_kind = {ctypes.c_void_p: "pointer", ctypes.c_size_t: "size", ctypes.c_int64: "int64",
               ctypes.c_int: "int", _lib.ff2: "ff2", ctypes.c_char_p: "pointer", None: "void"}
    for name, (ret, params) in protos.items():
        res, args = _lib.SIGNATURES[name]
        assert len(args) == len(params), (name, params)
        got = [py_kind.get(a, "pointer" if hasattr(a, "contents") or a.__name__.startswith("LP_") else "?")
               for a in args]
        want = [_ctypes_kind(p) for p in params]
        assert got == want, (name, got, want)
        assert py_kind[res] == _ctypes_kind(ret), (name, res, ret)
