"""Replays of the CUDA reductions' documented combination order, built from
the oracle's Add22 / Mul22 array operators.

The oracle itself only defines the left-to-right accumulation; these helpers
re-order the same oracle operators the way the kernels document (include/ff.h,
ff_sum) so that a test can check a GPU reduction bit for bit, not just
within its error bound.  Used by the tests only.
"""
from __future__ import annotations

import numpy as np

import oracle

BLOCK = 256
WARPS = BLOCK // 32


def _add22(a, b):
    return oracle.add22(np.ascontiguousarray(a), np.ascontiguousarray(b))


def _warp_tree(v):
    """v: (..., 32, 2) lane values -> (..., 2), the shuffle-down tree lane 0
    computes (v_l = add22(v_l, v_{l+off}), off = 16 .. 1)."""
    v = v.copy()
    off = 16
    while off >= 1:
        lhs = v[..., :off, :].reshape(-1, 2)
        rhs = v[..., off:2 * off, :].reshape(-1, 2)
        v[..., :off, :] = _add22(lhs, rhs).reshape(v[..., :off, :].shape)
        off //= 2
    return v[..., 0, :]


def _block_tree(vals):
    """vals: (G, 256, 2) thread values -> (G, 2) block values."""
    G = vals.shape[0]
    w = _warp_tree(vals.reshape(G, WARPS, 32, 2))           # (G, 8, 2)
    off = WARPS // 2
    while off >= 1:
        lhs = w[:, :off, :].reshape(-1, 2)
        rhs = w[:, off:2 * off, :].reshape(-1, 2)
        w[:, :off, :] = _add22(lhs, rhs).reshape(G, off, 2)
        off //= 2
    return w[:, 0, :]


def reduce_replay(terms: np.ndarray, grid: int, head: int, vector: bool) -> np.ndarray:
    """The kernels' result for per-element float-float terms (x_i for the
    sum, Mul22(x_i, y_i) for the dot) -- bit for bit."""
    n = terms.shape[0]
    T = grid * BLOCK
    # per-thread ordered element lists
    if vector:
        nv = (n - head) // 2
        chunks_per_thread = -(-nv // T) if nv else 0
        seq = np.full((T, 2 * chunks_per_thread), -1, dtype=np.int64)
        for s in range(chunks_per_thread):
            c = np.arange(T) + s * T
            ok = c < nv
            seq[ok, 2 * s] = head + 2 * c[ok]
            seq[ok, 2 * s + 1] = head + 2 * c[ok] + 1
        pre = [0] if head == 1 else []
        post = [n - 1] if (n - head) % 2 == 1 else []
    else:
        per = -(-n // T) if n else 0
        seq = np.full((T, per), -1, dtype=np.int64)
        for s in range(per):
            i = np.arange(T) + s * T
            ok = i < n
            seq[ok, s] = i[ok]
        pre, post = [], []
    acc = np.zeros((T, 2), np.float32)
    for i in pre:
        acc[0] = _add22(acc[0:1], terms[i:i + 1])[0]
    for s in range(seq.shape[1]):
        idx = seq[:, s]
        ok = idx >= 0
        if ok.any():
            acc[ok] = _add22(acc[ok], terms[idx[ok]])
    for i in post:
        acc[0] = _add22(acc[0:1], terms[i:i + 1])[0]
    part = _block_tree(acc.reshape(grid, BLOCK, 2))
    if grid == 1:
        return part[0]
    acc2 = np.zeros((BLOCK, 2), np.float32)
    for b0 in range(0, grid, BLOCK):
        sl = part[b0:b0 + BLOCK]
        acc2[: sl.shape[0]] = _add22(acc2[: sl.shape[0]], sl)
    return _block_tree(acc2.reshape(1, BLOCK, 2))[0]
