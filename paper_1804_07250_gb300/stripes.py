"""One chain split across GPUs by rows: the bookkeeping of the exchange.

Within a pass every site of a colour class is updated independently, and a
site reads only the edges around it (Sec. 1.1.3, Sec. 2.2), so the state one
pass later depends on the rows within one of it.  A rank that owns the rows
[lo, hi) and also holds `halo` rows on each side can run `halo` passes alone:
after pass i the rows within halo - i of its stripe are still exact, so its
own rows are exact after `halo` passes.  It then sends its first and last
`halo` rows to the neighbouring ranks and receives theirs: one exchange per
`halo` passes, `halo` rows of every plane per seam and direction.  Random
numbers are keyed by the site's own coordinates and the absolute sweep, so
the result is the same on any number of ranks.

This module holds the partition, the schedule and the row exchange over
torch.distributed (point-to-point send/recv of canonical rows: NCCL between
GPUs, gloo on CPU); the per-rank update is whatever advances rows [slo, shi)
by a pass.  Stripe bounds are even, like the kernels' row pairs.
"""
from __future__ import annotations


def partition(height: int, world: int, halo: int):
    """Row bounds [lo, hi) of each rank: even, each stripe at least `halo`
    rows (so a rank's two boundary blocks never overlap), sizes as equal as
    that allows.  `height` is the number of vertex rows."""
    if world < 1 or halo < 1:
        raise ValueError("world and halo must be positive")
    rows = height + (height & 1)
    units = rows // 2
    if world > 1 and units < world * ((halo + 1) // 2):
        raise ValueError("%d rows cannot give %d stripes of %d rows" % (height, world, halo))
    base, extra = divmod(units, world)
    bounds, y = [], 0
    for r in range(world):
        n = 2 * (base + (1 if r < extra else 0))
        bounds.append((y, y + n))
        y += n
    return bounds


def local_rows(bounds, rank: int, halo: int, height: int):
    """Rows [slo, shi) rank `rank` holds: its stripe plus `halo` rows on each
    side that has a neighbour, clipped to the box."""
    lo, hi = bounds[rank]
    slo = lo - halo if rank > 0 else lo
    shi = hi + halo if rank < len(bounds) - 1 else hi
    return max(0, slo), min(height, shi)


def cycles(total_passes: int, halo: int):
    """Passes run between exchanges: full cycles of `halo`, then the rest."""
    out = [halo] * (total_passes // halo)
    if total_passes % halo:
        out.append(total_passes % halo)
    return out


def exchange(state, bounds, rank: int, halo: int, dist):
    """Refresh the halo rows of `state` (a tensor [planes][H][W] whose rows
    [lo - halo, hi + halo) this rank holds) from the neighbouring ranks: send
    the first and last `halo` own rows, receive the neighbours' into the
    halo.  Sends and receives are ordered so that no rank waits on another's
    send (even ranks send first)."""
    world = len(bounds)
    lo, hi = bounds[rank]
    H = state.shape[1]
    ops = []
    if rank > 0:
        ops.append(("send", rank - 1, lo, min(lo + halo, hi)))
        ops.append(("recv", rank - 1, max(0, lo - halo), lo))
    if rank < world - 1:
        ops.append(("send", rank + 1, max(lo, hi - halo), hi))
        ops.append(("recv", rank + 1, hi, min(H, hi + halo)))
    reqs = []
    for kind, peer, a, b in ops:
        blk = state[:, a:b, :].contiguous()
        if kind == "send":
            reqs.append((dist.isend(blk, peer), None, a, b))
        else:
            reqs.append((dist.irecv(blk, peer), blk, a, b))
    for req, blk, a, b in reqs:
        req.wait()
        if blk is not None:
            state[:, a:b, :] = blk
