"""Replays of the CUDA reductions' documented combination order, built from
the oracle's Add12 / Mul12 / Add22 / Mul22 array operators (and numpy's own
binary32 additions for the s-terms of Sum2 / Dot2).

The oracle itself only defines the left-to-right accumulation; these helpers
re-order the same operators the way the kernels document (include/ff.h,
ff_sum and ff_dot2) so that a test can check a GPU reduction bit for bit,
not just within its error bound.  Used by the tests only.
"""
from __future__ import annotations

import numpy as np

import oracle

BLOCK = 256
WARPS = BLOCK // 32
f32 = np.float32


class FFPolicy:
    """Add22 accumulation of float-float terms (ff_sum, ff_dot)."""
    E = 2   # values per 16-byte vector

    def zero(self, n):
        return np.zeros((n, 2), np.float32)

    def step(self, acc, t):
        return oracle.add22(np.ascontiguousarray(acc), np.ascontiguousarray(t))

    def combine(self, a, b):
        return oracle.add22(np.ascontiguousarray(a), np.ascontiguousarray(b))

    def finalize(self, a):
        return a


class Dot2Policy:
    """Compensated (p, s) accumulation of Ogita-Rump-Oishi's Sum2 / Dot2.
    Terms are (h, r) pairs: TwoProduct(x_i, y_i) for Dot2, (x_i, 0) for Sum2."""
    E = 4

    def zero(self, n):
        return np.zeros((n, 2), np.float32)

    def step(self, acc, t):
        pq = oracle.add12(np.ascontiguousarray(np.stack([acc[:, 0], t[:, 0]], 1)))
        s = (acc[:, 1] + (pq[:, 1] + t[:, 1]).astype(f32)).astype(f32)
        return np.stack([pq[:, 0], s], 1).astype(f32)

    def combine(self, a, b):
        pq = oracle.add12(np.ascontiguousarray(np.stack([a[:, 0], b[:, 0]], 1)))
        s = (a[:, 1] + (b[:, 1] + pq[:, 1]).astype(f32)).astype(f32)
        return np.stack([pq[:, 0], s], 1).astype(f32)

    def finalize(self, a):
        return oracle.add12(np.ascontiguousarray(a.reshape(1, 2)))[0]


def _warp_tree(pol, v):
    """v: (G*W, 32, 2) lane values -> (G*W, 2): the shuffle-down tree lane 0
    computes (v_l = combine(v_l, v_{l+off}), off = 16 .. 1)."""
    v = v.copy()
    off = 16
    while off >= 1:
        lhs = v[:, :off, :].reshape(-1, 2)
        rhs = v[:, off:2 * off, :].reshape(-1, 2)
        v[:, :off, :] = pol.combine(lhs, rhs).reshape(v.shape[0], off, 2)
        off //= 2
    return v[:, 0, :]


def _block_tree(pol, vals):
    """vals: (G, 256, 2) thread values -> (G, 2) block values."""
    G = vals.shape[0]
    w = _warp_tree(pol, vals.reshape(G * WARPS, 32, 2)).reshape(G, WARPS, 2)
    off = WARPS // 2
    while off >= 1:
        lhs = w[:, :off, :].reshape(-1, 2)
        rhs = w[:, off:2 * off, :].reshape(-1, 2)
        w[:, :off, :] = pol.combine(lhs, rhs).reshape(G, off, 2)
        off //= 2
    return w[:, 0, :]


def reduce_replay(terms: np.ndarray, grid: int, head: int, vector: bool, pol=None) -> np.ndarray:
    """The kernels' result for per-value terms (x_i for ff_sum, Mul22(x_i, y_i)
    for ff_dot; (h_i, r_i) for Sum2 / Dot2) -- bit for bit."""
    pol = pol or FFPolicy()
    E = pol.E
    n = terms.shape[0]
    T = grid * BLOCK
    if vector:
        nv = (n - head) // E
        per = -(-nv // T) if nv else 0
        seq = np.full((T, E * per), -1, dtype=np.int64)
        for s in range(per):
            c = np.arange(T) + s * T
            ok = c < nv
            for e in range(E):
                seq[ok, E * s + e] = head + E * c[ok] + e
        pre = list(range(head))
        post = list(range(head + nv * E, n))
    else:
        per = -(-n // T) if n else 0
        seq = np.full((T, per), -1, dtype=np.int64)
        for s in range(per):
            i = np.arange(T) + s * T
            ok = i < n
            seq[ok, s] = i[ok]
        pre, post = [], []
    acc = pol.zero(T)
    for i in pre:
        acc[0:1] = pol.step(acc[0:1], terms[i:i + 1])
    for s in range(seq.shape[1]):
        idx = seq[:, s]
        ok = idx >= 0
        if ok.any():
            acc[ok] = pol.step(acc[ok], terms[idx[ok]])
    for i in post:
        acc[0:1] = pol.step(acc[0:1], terms[i:i + 1])
    part = _block_tree(pol, acc.reshape(grid, BLOCK, 2))
    if grid == 1:
        return pol.finalize(part[0])
    acc2 = pol.zero(BLOCK)
    for b0 in range(0, grid, BLOCK):
        sl = part[b0:b0 + BLOCK]
        acc2[: sl.shape[0]] = pol.combine(acc2[: sl.shape[0]], sl)
    return pol.finalize(_block_tree(pol, acc2.reshape(1, BLOCK, 2))[0])
