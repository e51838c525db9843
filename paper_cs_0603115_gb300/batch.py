"""Batched float-float dot, AXPY, dot-adjoint and GEMV instances in one
persistent launch.

Thin wrapper over the C ABI's ff_batch_* entry points: a ``BatchPlan`` holds
the native plan (instance records and tile list on the device), its
workspace, and optionally an instantiated CUDA graph of its run.  ``autotune``
times every candidate launch configuration through ``ff_batch_autotune`` and
caches the winner in a JSON file keyed by kernel, SM count, workload size
bucket and library build id.
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import torch

from . import _lib
from ._lib import ff2, ff_batch_instance, ff_tune

DOT = 0
AXPY = 1
DOT_GRAD = 2
GEMV = 3
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "ff_gb300", "autotune.json")


def _check_instance(i, kind, x, y, out, out2, dout, cur):
    """The plan reads and writes through plain pointers: every tensor must be
    a contiguous float32 tensor on the current device with the extent the
    instance kind implies."""
    def ok(t, numel=None):
        return (t is not None and t.is_cuda and t.device.index == cur and t.dtype == torch.float32
                and t.is_contiguous() and (numel is None or t.numel() == numel))
    if kind == GEMV:
        good = (ok(x) and x.dim() == 3 and x.shape[2] == 2 and ok(y, 2 * x.shape[1]) and ok(out, 2 * x.shape[0]))
    elif kind == DOT:
        good = ok(x) and ok(y, x.numel()) and ok(out, 2)
    elif kind == AXPY:
        good = ok(x) and ok(y, x.numel()) and ok(out, x.numel())
    elif kind == DOT_GRAD:
        good = ok(x) and ok(y, x.numel()) and ok(out, x.numel()) and ok(out2, x.numel()) and ok(dout, 2)
    else:
        raise ValueError(f"instance {i}: unknown kind {kind}")
    if not good:
        raise ValueError(f"instance {i} (kind {kind}): tensors must be contiguous float32 on cuda:{cur} "
                         "with the sizes of that kind")


def make_instances(specs) -> ctypes.Array:
    """specs: iterable of (kind, x, y, out, alpha) or (kind, x, y, out, alpha,
    out2, dout) with x, y, out CUDA float-float tensors (out is a (2,) tensor
    for DOT), alpha a (hi, lo) pair (AXPY only), and for DOT_GRAD out = dx,
    out2 = dy and dout a (2,) device tensor.  For GEMV, x is the (m, n, 2)
    row-major matrix, y the (n, 2) vector and out the (m, 2) result."""
    specs = list(specs)
    arr = (ff_batch_instance * len(specs))()
    cur = torch.cuda.current_device()
    for i, spec in enumerate(specs):
        kind, x, y, out, alpha = spec[:5]
        out2 = spec[5] if len(spec) > 5 else None
        dout = spec[6] if len(spec) > 6 else None
        _check_instance(i, kind, x, y, out, out2, dout, cur)
        arr[i].kind = kind
        arr[i].reserved = 0
        if kind == GEMV:
            arr[i].n = x.shape[1]
            arr[i].m = x.shape[0]
            arr[i].lda = x.shape[1]
        else:
            arr[i].n = x.numel() // 2
        arr[i].x = x.data_ptr()
        arr[i].y = y.data_ptr()
        arr[i].out = out.data_ptr()
        arr[i].out2 = out2.data_ptr() if out2 is not None else None
        arr[i].dout = dout.data_ptr() if dout is not None else None
        a = alpha if alpha is not None else (0.0, 0.0)
        arr[i].alpha = ff2(float(a[0]), float(a[1]))
    return arr


class BatchPlan:
    def __init__(self, instances: ctypes.Array, tune: tuple | None = None, device=None):
        L = _lib.load()
        self.instances = instances
        self.count = len(instances)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        handle = ctypes.c_void_p()
        t = ff_tune(*tune) if tune is not None else None
        _lib.call("ff_batch_plan_create", instances, self.count, ctypes.byref(t) if t is not None else None,
                  ctypes.byref(handle))
        self.handle = handle
        nbytes = L.ff_batch_workspace_bytes(handle)
        self.ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        self.graph = None
        info = ff_tune()
        ntiles = ctypes.c_int64()
        grid = ctypes.c_uint()
        _lib.call("ff_batch_plan_info", handle, ctypes.byref(info), ctypes.byref(ntiles), ctypes.byref(grid))
        self.tune = (info.block, info.pairs_per_thread, info.blocks_per_sm, info.unroll)
        self.ntiles = ntiles.value
        self.grid = grid.value

    def run(self):
        """One memset + one persistent kernel on the current stream."""
        _lib.call("ff_batch_run", self.handle, self.ws.data_ptr(), self.ws.numel(),
                  torch.cuda.current_stream().cuda_stream)

    def capture(self):
        """Instantiate a CUDA graph of run()."""
        if self.graph is None:
            g = ctypes.c_void_p()
            _lib.call("ff_batch_graph_create", self.handle, self.ws.data_ptr(), self.ws.numel(), ctypes.byref(g))
            self.graph = g
        return self

    def launch(self):
        """Replay the captured graph on the current stream."""
        if self.graph is None:
            self.capture()
        _lib.call("ff_batch_graph_launch", self.graph, torch.cuda.current_stream().cuda_stream)

    def close(self):
        L = _lib.load()
        if self.graph is not None:
            torch.cuda.synchronize(self.device)
            L.ff_batch_graph_destroy(self.graph)
            self.graph = None
        if self.handle is not None:
            torch.cuda.synchronize(self.device)
            L.ff_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _cache_key(instances) -> str:
    L = _lib.load()
    total = sum(int(instances[i].n) for i in range(len(instances)))
    sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    bucket = int(math.log2(total)) if total > 0 else 0
    cbucket = int(math.log2(len(instances))) if len(instances) > 0 else 0
    return f"ff_batch|sm{sm}|v2^{bucket}|c2^{cbucket}|{L.ff_build_id().decode()}"


def autotune(instances, reps: int = 3, cache_path: str | None = DEFAULT_CACHE, force: bool = False):
    """Pick (block, pairs_per_thread, blocks_per_sm, unroll) for these instances.

    Looks the workload's key up in the JSON cache first; otherwise times
    every candidate natively (the instances' outputs are overwritten) and
    stores the winner.  Returns (tune, ms_per_run or None if cached)."""
    key = _cache_key(instances)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if not force and key in cache:
        t = cache[key]["tune"]
        return tuple(t), None
    L = _lib.load()
    nbytes = L.ff_batch_autotune_workspace_bytes(instances, len(instances))
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
    best = ff_tune()
    ms = ctypes.c_float()
    _lib.call("ff_batch_autotune", instances, len(instances), ws.data_ptr(), ws.numel(),
              torch.cuda.current_stream().cuda_stream, reps, ctypes.byref(best), ctypes.byref(ms))
    tune = (best.block, best.pairs_per_thread, best.blocks_per_sm, best.unroll)
    if cache_path:
        cache[key] = {"tune": list(tune), "ms": ms.value}
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return tune, ms.value


def candidates():
    L = _lib.load()
    n = L.ff_batch_tune_candidates(None, 0)
    arr = (ff_tune * n)()
    L.ff_batch_tune_candidates(arr, n)
    return [(c.block, c.pairs_per_thread, c.blocks_per_sm, c.unroll) for c in arr]
