"""Host models of three exact shortcuts the CUDA path takes, checked against
the plain rule they replace (no GPU, no oracle: these pin the reasoning the
kernels rely on, on random inputs).

- The propagation engine's overflow radix queue: with every key at most the
  base, a lower bucket holds higher keys; pushes below the last pop and pops
  with refiling give the pops of an ordinary max-priority queue.
- The local-order rounds: popping the longest prefix of the queue's next keys
  in which no key queued by an earlier candidate comes before a later one
  gives the one-by-one visiting order of a priority propagation.
- The bounded cut search: a piece of R minus a candidate that is exhausted
  without reaching s (or another search's piece) proves that removing the
  candidate disconnects R.
"""
import heapq
import random

import pytest

# ---- radix queue (propagation engine overflow) ----


def bucket(base, key):
    return 0 if key == base else (base ^ key).bit_length()


def test_lower_buckets_hold_higher_keys():
    rng = random.Random(1)
    for _ in range(2000):
        base = rng.randrange(1, 1 << 31)
        keys = [rng.randrange(0, base + 1) for _ in range(20)]
        for a in keys:
            for b in keys:
                if bucket(base, a) < bucket(base, b):
                    assert a > b
        # refiling a bucket under its highest key sends its entries to lower buckets
        by = {}
        for k in keys:
            by.setdefault(bucket(base, k), []).append(k)
        for bk, ks in by.items():
            if bk == 0:
                continue
            nb = max(ks)
            assert all(bucket(nb, k) < bk for k in ks)


class RadixQ:
    def __init__(self, base=(1 << 31) - 1):
        self.base = base
        self.b = [[] for _ in range(33)]

    def push(self, k):
        assert k <= self.base
        self.b[bucket(self.base, k)].append(k)

    def __len__(self):
        return sum(map(len, self.b))

    def top(self):
        for lst in self.b:
            if lst:
                return max(lst)
        return None

    def pop(self):
        i = next(j for j, lst in enumerate(self.b) if lst)
        if i > 0 and len(self.b[i]) == 1:
            return self.b[i].pop()
        if i > 0:
            ks, self.b[i] = self.b[i], []
            self.base = max(ks)
            for k in ks:
                self.push(k)
        return self.b[0].pop()


@pytest.mark.parametrize("seed", range(6))
def test_radix_queue_pops_like_a_max_heap_under_monotone_pushes(seed):
    rng = random.Random(seed)
    q, h = RadixQ(), []
    last = rng.randrange(1 << 20, 1 << 27)
    for k in (rng.randrange(0, last) for _ in range(50)):
        q.push(k)
        heapq.heappush(h, -k)
    pops = 0
    while h and pops < 3000:
        a, b = q.pop(), -heapq.heappop(h)
        assert a == b
        last = a
        pops += 1
        for _ in range(rng.randrange(0, 4)):        # what a pop queues is below it
            if last > 0:
                k = rng.randrange(0, last)
                q.push(k)
                heapq.heappush(h, -k)
    assert len(q) == len(h)


def test_absorbing_a_queue_keeps_the_order():
    rng = random.Random(9)
    for _ in range(200):
        v = rng.randrange(1 << 10, 1 << 20)           # the saddle both classes popped last
        a, b = RadixQ(rng.randrange(v, 1 << 21)), RadixQ(rng.randrange(v, 1 << 21))
        ka = [rng.randrange(0, v) for _ in range(rng.randrange(0, 40))]
        kb = [rng.randrange(0, v) for _ in range(rng.randrange(0, 40))]
        for k in ka:
            a.push(k)
        for k in kb:
            b.push(k)
        big, small = (a, b) if len(a) >= len(b) else (b, a)
        for lst in small.b:
            for k in lst:
                big.push(k)
        got = [big.pop() for _ in range(len(big))]
        assert got == sorted(ka + kb, reverse=True)


# ---- rounds of the key-space local-order propagation ----


def random_graph(rng, n, p):
    adj = [set() for _ in range(n)]
    order = list(range(n))
    rng.shuffle(order)
    for i in range(1, n):                            # connected: a random tree first
        j = order[rng.randrange(0, i)]
        adj[order[i]].add(j)
        adj[j].add(order[i])
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < p:
                adj[i].add(j)
                adj[j].add(i)
    return [sorted(s) for s in adj]


def flood_one_by_one(adj, key, seeds, maxf):
    sign = -1 if maxf else 1
    h = [(sign * key[i], i) for i in seeds]
    heapq.heapify(h)
    vis = set(seeds)
    out = []
    while h:
        _, i = heapq.heappop(h)
        out.append(i)
        for j in adj[i]:
            if j not in vis:
                vis.add(j)
                heapq.heappush(h, (sign * key[j], j))
    return out


def flood_in_rounds(adj, key, seeds, maxf, width=32):
    """The rule of the warp tier: candidates are the queue's next `width` keys
    in pop order; candidate j is popped in this round when every candidate
    before it is and no not-yet-queued neighbour of those comes before it."""
    better = (lambda x, y: x > y) if maxf else (lambda x, y: x < y)
    queued = set(seeds)                              # queued or popped
    queue = set(seeds)
    out = []
    while queue:
        cands = sorted(queue, key=lambda i: -key[i] if maxf else key[i])[:width]
        best_new = None
        pref = 0
        for c in cands:
            if best_new is not None and better(best_new, key[c]):
                break
            pref += 1
            for j in adj[c]:
                if j not in queued and (best_new is None or better(key[j], best_new)):
                    best_new = key[j]
        for c in cands[:pref]:
            queue.discard(c)
            out.append(c)
            for j in adj[c]:
                if j not in queued:
                    queued.add(j)
                    queue.add(j)
    return out


@pytest.mark.parametrize("maxf", [True, False])
def test_rounds_visit_in_the_one_by_one_order(maxf):
    rng = random.Random(3 + maxf)
    for it in range(300):
        n = rng.randrange(2, 90)
        adj = random_graph(rng, n, rng.choice([0.0, 0.02, 0.08]))
        key = list(range(n))
        rng.shuffle(key)
        seeds = rng.sample(range(n), rng.randrange(1, min(n, 4) + 1))
        width = rng.choice([2, 5, 32])
        assert flood_in_rounds(adj, key, seeds, maxf, width) == flood_one_by_one(adj, key, seeds, maxf), it


# ---- bounded cut search (minus-infinity candidates) ----


def connected_without(adj, a, s):
    seen = {s}
    stack = [s]
    while stack:
        u = stack.pop()
        for w in adj[u]:
            if w != a and w not in seen:
                seen.add(w)
                stack.append(w)
    return len(seen) == len(adj) - 1


def cuts_model(adj, a, s, budget):
    """The warp tier's search: from each neighbour of a (but s) over R minus
    a; a search that ends within the budget without reaching s or a vertex an
    earlier search reached has found a piece cut off by a."""
    mark = {}
    for t, b0 in enumerate(x for x in adj[a] if x != s):
        if b0 in mark:
            continue
        mark[b0] = t
        q, head, reach, over = [b0], 0, False, False
        while head < len(q) and not reach and not over:
            i = q[head]
            head += 1
            for j in adj[i]:
                if j == a:
                    continue
                if j == s:
                    reach = True
                    continue
                if j in mark:
                    if mark[j] != t:
                        reach = True
                    continue
                mark[j] = t
                q.append(j)
                over = len(q) > budget
        if not reach and not over:
            return True
    return False


def test_a_found_piece_proves_the_cut():
    rng = random.Random(11)
    found = 0
    for _ in range(1500):
        n = rng.randrange(3, 60)
        adj = random_graph(rng, n, rng.choice([0.0, 0.03, 0.1]))
        s = rng.randrange(n)
        a = rng.choice([i for i in range(n) if i != s])
        for budget in (2, 8, 64):
            if cuts_model(adj, a, s, budget):
                assert not connected_without(adj, a, s)
                found += 1
    assert found > 100
