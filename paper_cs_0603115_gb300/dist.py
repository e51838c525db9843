"""Sharded float-float reductions over several GPUs (one process per GPU).

A dot product or sum sharded over ranks has one real exchange step: every
rank reduces its contiguous shard with the library's kernel, the ranks
all-gather their 8-byte float-float partials, and every rank combines the
gathered partials in rank order with Add22 (the library's ff_sum on the
rank-ordered vector of partials), so all ranks hold the same bits.  A
collective sum (e.g. NCCL's SUM) cannot be used: it would add the high and
the low parts separately.

GEMV needs no exchange when A is sharded by rows (each rank owns its rows of
Y); its adjoint dX = A^T dY does: every rank computes the (k, n) partial of
its rows.  The columns are cut into one contiguous block per rank; rank b
receives every rank's partial of block b (point-to-point sends), adds them
in rank order with Add22 (ff_add) and the combined blocks are all-gathered.
Each column sees the same rank-ordered Add22 sequence as if every rank
combined all partials, for 1/world of the exchanged bytes and of the
additions.

The compute functions are arguments (defaulting to the library's kernels)
so that the exchange logic can be exercised on CPU-only ranks with stand-ins.
"""
from __future__ import annotations

import torch


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous shard [lo, hi) of n items for `rank` of `world` (the first
    n % world ranks get one more item)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def _all_gather_rows(t: torch.Tensor, group=None) -> torch.Tensor:
    """(world, *t.shape): every rank's tensor, in rank order."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t.contiguous(), group=group)
    return torch.stack(parts)


def combine_partials(parts: torch.Tensor, sum_fn=None) -> torch.Tensor:
    """Rank-ordered Add22 combination of (world, 2) float-float partials."""
    if sum_fn is None:
        from . import sum as sum_fn
    return sum_fn(parts.contiguous())


def sharded_dot(x_local: torch.Tensor, y_local: torch.Tensor, group=None, dot_fn=None, sum_fn=None):
    """Float-float dot product of vectors sharded over the ranks of `group`
    (each rank passes its own contiguous shard).  Returns the (2,) result,
    bit-identical on every rank."""
    if dot_fn is None:
        from . import dot as dot_fn
    local = dot_fn(x_local, y_local)
    parts = _all_gather_rows(local.reshape(2), group)
    return combine_partials(parts, sum_fn)


def sharded_sum(x_local: torch.Tensor, group=None, sum_fn=None):
    """Float-float sum of a vector sharded over the ranks of `group`."""
    if sum_fn is None:
        from . import sum as sum_fn
    local = sum_fn(x_local)
    parts = _all_gather_rows(local.reshape(2), group)
    return combine_partials(parts, sum_fn)


def _exchange(send: list, recv: list, group=None) -> None:
    """recv[r] = rank r's send[this rank] for every other rank r (point to
    point; empty blocks are neither sent nor received)."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    ops = []
    for r in range(len(send)):
        if r == rank:
            continue
        peer = dist.get_global_rank(group, r) if group is not None else r
        if send[r].numel():
            ops.append(dist.P2POp(dist.isend, send[r], peer, group))
        if recv[r].numel():
            ops.append(dist.P2POp(dist.irecv, recv[r], peer, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def sharded_gemv_t(A_local: torch.Tensor, dY_local: torch.Tensor, group=None, gemv_t_fn=None, add_fn=None):
    """dX = A^T dY for A sharded by rows: A_local (m_r, n, 2) and dY_local
    (k, m_r, 2) are this rank's rows.  Returns the (k, n, 2) dX, equal on every
    rank: for every column the per-rank partials are added in rank order with
    Add22.  Exchange: reduce-scatter by column block (each rank combines the
    block shard_range(n, rank, world) of every rank's partial), then an
    all-gather of the combined blocks."""
    import torch.distributed as dist
    if gemv_t_fn is None:
        from . import gemv_t as gemv_t_fn
    if add_fn is None:
        from . import add as add_fn
    local = gemv_t_fn(A_local, dY_local)
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    k, n = local.shape[0], local.shape[1]
    if world == 1 or n == 0:
        return local
    spans = [shard_range(n, b, world) for b in range(world)]
    lo, hi = spans[rank]
    send = [local[:, a:b].contiguous() for a, b in spans]
    recv = [send[r] if r == rank else torch.empty((k, hi - lo, 2), dtype=local.dtype, device=local.device)
            for r in range(world)]
    _exchange(send, recv, group)
    acc = recv[0]
    for r in range(1, world):
        acc = add_fn(acc.contiguous(), recv[r].contiguous())
    width = max(b - a for a, b in spans)
    mine = torch.zeros((k, width, 2), dtype=local.dtype, device=local.device)
    mine[:, :hi - lo] = acc
    blocks = _all_gather_rows(mine, group)
    return torch.cat([blocks[b, :, :spans[b][1] - spans[b][0]] for b in range(world)], dim=1).contiguous()


def partition_instances(nbytes, world: int) -> list[list[int]]:
    """Byte-balanced split of batched instances over `world` ranks: instances
    in decreasing order of bytes, each to the rank with the fewest bytes so
    far (ties: the lowest rank); every rank's list is returned in increasing
    instance order.  The busiest rank carries at most the average plus the
    largest instance."""
    import heapq
    order = sorted(range(len(nbytes)), key=lambda i: (-int(nbytes[i]), i))
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + int(nbytes[i]), r))
    return [sorted(p) for p in parts]
