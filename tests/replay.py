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


def gemv_rows8_replay(A, x, vec: bool):
    """Rows of a batched GEMV reduced by eight lanes each (ff_batch.cu, the
    GEMV-rows tile): lane l of the row takes the two-value chunks l + 16i into
    its first and l + 8 + 16i into its second accumulator while both fit, a
    leftover chunk l + 16i into the first; adds the two; with an odd length,
    lane 0 adds the last term; then the shuffle-down Add22 tree over offsets
    4, 2, 1.  Without 16-byte access (vec False) lane l takes the terms
    l + 8i into one accumulator.  A: (m, n, 2), x: (n, 2); returns (m, 2)."""
    A = np.ascontiguousarray(A, np.float32)
    x = np.ascontiguousarray(x, np.float32)
    m, n = A.shape[0], A.shape[1]
    terms = oracle.mul22(A.reshape(-1, 2), np.tile(x, (m, 1))).reshape(m, n, 2) if m * n else np.zeros((m, n, 2), f32)
    add = lambda a, b: oracle.add22(np.ascontiguousarray(a), np.ascontiguousarray(b))
    acc = np.zeros((m, 8, 2), f32)
    if vec:
        acc1 = np.zeros((m, 8, 2), f32)
        nch = n // 2
        for l in range(8):
            c = l
            while c + 8 < nch:
                acc[:, l] = add(add(acc[:, l], terms[:, 2 * c]), terms[:, 2 * c + 1])
                acc1[:, l] = add(add(acc1[:, l], terms[:, 2 * (c + 8)]), terms[:, 2 * (c + 8) + 1])
                c += 16
            while c < nch:
                acc[:, l] = add(add(acc[:, l], terms[:, 2 * c]), terms[:, 2 * c + 1])
                c += 8
            acc[:, l] = add(acc[:, l], acc1[:, l])
        if n & 1:
            acc[:, 0] = add(acc[:, 0], terms[:, n - 1])
    else:
        for l in range(8):
            for j in range(l, n, 8):
                acc[:, l] = add(acc[:, l], terms[:, j])
    for off in (4, 2, 1):
        for l in range(off):
            acc[:, l] = add(acc[:, l], acc[:, l + off])
    return acc[:, 0]


def gemv_warp_replay(A, X, vec: bool):
    """ff_gemv's order (include/ff.h): row r is reduced by a warp; lane l
    accumulates, from (0, 0), its two-value chunks l, l + 32, l + 64, ...
    (vec) or its values l, l + 32, ... (not vec) with Add22(acc, Mul22(A, X)),
    then the shuffle-down Add22 tree over offsets 16 .. 1.  A: (m, n, 2);
    X: (k, n, 2); returns Y as (k, m, 2)."""
    A = np.ascontiguousarray(A, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    m, n = A.shape[0], A.shape[1]
    k = X.shape[0]
    Y = np.zeros((k, m, 2), f32)
    add = lambda a, b: oracle.add22(np.ascontiguousarray(a), np.ascontiguousarray(b))
    for c in range(k):
        terms = oracle.mul22(A.reshape(-1, 2), np.tile(X[c], (m, 1))).reshape(m, n, 2) if m * n else np.zeros((m, n, 2), f32)
        acc = np.zeros((m, 32, 2), f32)
        for l in range(32):
            if vec:
                idx = [j for t in range(l, n // 2, 32) for j in (2 * t, 2 * t + 1)]
            else:
                idx = list(range(l, n, 32))
            for j in idx:
                acc[:, l] = add(acc[:, l], terms[:, j])
        for off in (16, 8, 4, 2, 1):
            for l in range(off):
                acc[:, l] = add(acc[:, l], acc[:, l + off])
        Y[c] = acc[:, 0]
    return Y


def gemv_t_replay(A, dY, row_blocks: int):
    """ff_gemv_t's order (include/ff.h): rows cut into row_blocks blocks of
    ceil(m / row_blocks) rows; within a block every column accumulates its
    rows in order from (0, 0) (the oracle's own gemv_t on the block); the
    blocks' partials are added in block order starting from the first.
    A: (m, n, 2); dY: (k, m, 2); returns dX as (k, n, 2)."""
    A = np.ascontiguousarray(A, np.float32)
    dY = np.ascontiguousarray(dY, np.float32)
    m = A.shape[0]
    rpb = -(-m // row_blocks) if m else 0
    parts = []
    for b in range(row_blocks):
        r0, r1 = min(m, b * rpb), min(m, (b + 1) * rpb)
        parts.append(oracle.gemv_t(np.ascontiguousarray(A[r0:r1]), np.ascontiguousarray(dY[:, r0:r1])))
    acc = parts[0]
    for p in parts[1:]:
        acc = oracle.add22(acc.reshape(-1, 2), p.reshape(-1, 2)).reshape(acc.shape)
    return acc


def _batch_block_tree(acc, block):
    """The batched kernel's block reduction: a shuffle-down Add22 tree
    (offsets 16 .. 1) inside every warp, then warp 0 combines the warps'
    results (lanes >= warps hold (0, 0)) with offsets warps/2 .. 1."""
    add = lambda a, b: oracle.add22(np.ascontiguousarray(a), np.ascontiguousarray(b))
    w = block // 32
    v = acc.reshape(w, 32, 2).copy()
    for off in (16, 8, 4, 2, 1):
        for l in range(off):
            v[:, l] = add(v[:, l], v[:, l + off])
    s = v[:, 0].copy()
    off = w // 2
    while off > 0:
        for l in range(off):
            s[l] = add(s[l:l + 1], s[l + off:l + off + 1])[0]
        off //= 2
    return s[0]


def batch_dot_replay(x, y, block: int, ppt: int, vec):
    """A DOT instance of the batched kernel (ff_batch.cu): tiles of
    block x ppt values; in a tile, thread t accumulates from (0, 0) the
    two-value chunks t, t + block, ... (vec 1 or True: 16-byte access; with an
    odd tile length thread 0 then adds the last value), or thread 0 first
    adds the tile's first value on its own and the chunks start one value
    later (vec 2: x and y both 8 bytes past a 16-byte boundary), or the
    values t, t + block, ... (vec 0 or False), each term Add22(acc,
    Mul22(x_i, y_i)); the block tree combines the threads; one tile writes
    its value, several tiles are combined by the last one: thread p adds the
    tile partials p, p + block, ... from (0, 0), then the block tree.
    Returns the (2,) result."""
    add = lambda a, b: oracle.add22(np.ascontiguousarray(a), np.ascontiguousarray(b))
    mode = int(vec)
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    n = x.shape[0]
    tile = block * ppt
    nt = max(1, -(-n // tile))
    terms = oracle.mul22(x, y) if n else np.zeros((0, 2), f32)
    parts = []
    for t in range(nt):
        s0, s1 = t * tile, min((t + 1) * tile, n)
        T = terms[s0:s1]
        acc = np.zeros((block, 2), f32)
        tid = np.arange(block)
        if mode:
            h = 1 if (mode == 2 and s1 > s0) else 0
            if h:
                acc[0] = add(acc[0:1], T[0:1])[0]
            T = T[h:]
            ln = s1 - s0 - h
            nch = ln // 2
            for j in range(ppt // 2):
                c = tid + j * block
                ok = c < nch
                if ok.any():
                    cc = c[ok]
                    acc[ok] = add(add(acc[ok], T[2 * cc]), T[2 * cc + 1])
            if ln & 1:
                acc[0] = add(acc[0:1], T[ln - 1:ln])[0]
        else:
            ln = s1 - s0
            for j in range(ppt):
                i = tid + j * block
                ok = i < ln
                if ok.any():
                    acc[ok] = add(acc[ok], T[i[ok]])
        parts.append(_batch_block_tree(acc, block))
    if nt == 1:
        return parts[0]
    P = np.array(parts, f32)
    acc = np.zeros((block, 2), f32)
    for p in range(nt):
        acc[p % block] = add(acc[p % block:p % block + 1], P[p:p + 1])[0]
    return _batch_block_tree(acc, block)
