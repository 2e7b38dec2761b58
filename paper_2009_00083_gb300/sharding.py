"""Batches and served requests spread over ranks by field (one process per
GPU).  Fields are independent units, so there is no collective on the data
path: each rank simplifies its own share, and only small per-field results
(status, statistics, output hashes) travel to the other ranks afterwards.

shard_fields(sizes, world)   deterministic partition of field indices over
                              ranks: largest field first, each to the rank
                              with the fewest vertices so far (lowest rank on
                              ties), so every rank computes the same partition
                              without talking to the others.
route_requests(n, world)     served request i goes to rank i mod world (the
                              arrival order is the only thing every rank knows).
gather_results(local, world, dist)   the per-field results of all ranks, in
                              field order (all_gather_object; world 1: local).
"""
from __future__ import annotations


def shard_fields(sizes, world):
    """Index lists (ascending) of the fields each rank simplifies."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += int(sizes[i])
    return [sorted(p) for p in parts]


def route_requests(n, world):
    """Request indices each rank serves (round robin in arrival order)."""
    return [list(range(r, n, world)) for r in range(world)]


def gather_results(local, world, dist=None):
    """local: {field index: result} of this rank.  Returns the results of every
    rank as one list in field order (every rank gets the same list)."""
    if world == 1 or dist is None:
        merged = dict(local)
    else:
        parts = [None] * world
        dist.all_gather_object(parts, dict(local))
        merged = {}
        for p in parts:
            for k, v in p.items():
                if k in merged:
                    raise RuntimeError(f"field {k} was simplified by two ranks")
                merged[k] = v
    return [merged[k] for k in sorted(merged)]


def run_sharded(sizes, simplify, rank, world, dist=None):
    """Runs simplify(i) for this rank's fields and gathers every field's
    result in field order.  simplify returns a small picklable result."""
    mine = shard_fields(sizes, world)[rank]
    local = {i: simplify(i) for i in mine}
    return gather_results(local, world, dist)
