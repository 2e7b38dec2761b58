"""Brute-force checkers written directly from the definitions (numpy / plain
Python), independent of the oracle's C code and of the CUDA library."""
from __future__ import annotations

from collections import deque

import numpy as np


def offsets(ndim):
    """Freudenthal neighbour offsets: the non-zero vectors of {0,1}^d and their negatives."""
    out = []
    for m in range(1, 1 << ndim):
        out.append(tuple((m >> b) & 1 for b in range(ndim)))
    out += [tuple(-c for c in o) for o in out]
    return out


def xyz_shape(shape):
    """(X, Y[, Z]) from the C-ordered array shape."""
    return tuple(reversed(shape))


def neighbours(shape, v):
    dims = xyz_shape(shape)
    nd = len(dims)
    coords = []
    r = v
    for d in dims:
        coords.append(r % d)
        r //= d
    out = []
    for o in offsets(nd):
        c = [coords[i] + o[i] for i in range(nd)]
        if all(0 <= c[i] < dims[i] for i in range(nd)):
            idx = 0
            mul = 1
            for i in range(nd):
                idx += c[i] * mul
                mul *= dims[i]
            out.append(idx)
    return out


def neighbour_table(shape):
    n = int(np.prod(shape))
    return [neighbours(shape, v) for v in range(n)]


def extrema(order, nbr):
    """(minima, maxima) of an injective order on the vertices (brute force)."""
    o = order.reshape(-1)
    mins, maxs = [], []
    for v in range(o.size):
        if all(o[u] > o[v] for u in nbr[v]):
            mins.append(v)
        if all(o[u] < o[v] for u in nbr[v]):
            maxs.append(v)
    return set(mins), set(maxs)


def component(nbr, start, allowed):
    """Vertices reachable from start through `allowed` (a boolean array)."""
    seen = {start}
    dq = deque([start])
    while dq:
        v = dq.popleft()
        for u in nbr[v]:
            if allowed[u] and u not in seen:
                seen.add(u)
                dq.append(u)
    return seen


def brute_regions(order, nbr, auth_max):
    """Regions of a maxima pass straight from the definition: vertex u is moved
    iff the component of {O >= O(u)} holding u has no authorized maximum; its
    saddle is the highest vertex s below u such that the component of
    {O >= O(s)} holding u has one.  Returns {u: saddle}."""
    o = order.reshape(-1)
    n = o.size
    perm = np.argsort(o)
    _, maxs = extrema(order, nbr)
    protect = {w for w in maxs if auth_max[w]}   # authorized ids that are not maxima are ignored
    out = {}
    for u in range(n):
        for lam in range(o[u], -1, -1):
            comp = component(nbr, u, o >= lam)
            if comp & protect:
                if lam != o[u]:
                    out[u] = int(perm[lam])
                break
    return out


def is_permutation(a):
    a = np.asarray(a).reshape(-1)
    return np.array_equal(np.sort(a), np.arange(a.size))
