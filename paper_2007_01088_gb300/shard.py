"""Sharding of the triple loop over ranks (one process per GPU).

The occupied triples i >= j >= k are independent units of work (Algorithm 1);
each contributes additively to Omega1, Omega2 and E_T.  A rank evaluates its
share through ``Context.set_triples`` and the partial results are summed with
one all-reduce per output at the end (the only exchange step of the path).
Shares are balanced by permutation weight (6 for distinct indices, 3 for a
repeated one; i = j = k contributes nothing).
"""
from __future__ import annotations

import heapq


def triples_with_weights(no: int):
    out = []
    for i in range(no):
        for j in range(i + 1):
            for k in range(j + 1):
                if i == j == k:
                    continue
                out.append(((i, j, k), 6 if (i != j and j != k) else 3))
    return out


def triple_partition(no: int, world: int, rank: int):
    """The triples of `rank` among `world` ranks: greedy longest-processing-
    time assignment by weight (every rank computes the same partition)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for t, w in sorted(triples_with_weights(no), key=lambda x: -x[1]):
        load, r = heapq.heappop(heap)
        parts[r].append(t)
        heapq.heappush(heap, (load + w, r))
    return sorted(parts[rank], reverse=True)


def omega_sharded(ctx, prec, out, group=None):
    """Sharded residual: this rank's triples, then a sum all-reduce of
    (Omega1, Omega2, E_T) over the process group.  `out` holds torch tensors:
    on the device for a device-pointer context (NCCL), in host memory for a
    host-pointer context (gloo).  The context is left restricted to this
    rank's triples."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    part = triple_partition(ctx.no, world, rank)
    if part:
        ctx.set_triples(part)
        ctx.omega(prec, out=out)
    else:
        for x in out:
            x.zero_()
    for x in out:
        dist.all_reduce(x, group=group)
    return out
