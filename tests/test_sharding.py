"""Batches and served requests sharded by field over ranks (no collective
on the data path).  The partition is checked on its own; the whole sharded
run is checked on two gloo ranks on the CPU, each simplifying its share of a
small mixed batch with the oracle as the per-field function: the gathered
results equal a single-process run."""
import os
import socket

import numpy as np
import pytest

from paper_2009_00083_gb300 import sharding as S

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def test_partition_is_disjoint_complete_balanced_and_deterministic():
    rng = np.random.default_rng(3)
    sizes = [int(x) for x in np.exp(rng.uniform(np.log(64 ** 2), np.log(160 ** 3), 256))]
    for world in (1, 2, 3, 4, 8):
        parts = S.shard_fields(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        assert parts == S.shard_fields(list(sizes), world)
        loads = [sum(sizes[i] for i in p) for p in parts]
        # largest-first greedy: no rank exceeds the mean by more than the largest field
        assert max(loads) - sum(loads) / world <= max(sizes)
    assert S.shard_fields([5, 4, 3, 3], 2) == [[0, 3], [1, 2]]
    assert S.route_requests(7, 3) == [[0, 3, 6], [1, 4], [2, 5]]


def _specs():
    from paper_2009_00083_gb300 import workloads as W

    rng = np.random.default_rng(9)
    out = []
    for k in range(9):
        shape = (int(rng.integers(12, 40)), int(rng.integers(12, 40))) if k % 2 else \
            tuple(int(rng.integers(6, 14)) for _ in range(3))
        out.append((shape, 8, 0.05, 100 + k))
    return out, W


def _simplify_one(i):
    import oracle

    specs, W = _specs()
    shape, K, noise, seed = specs[i]
    f = W.gaussian_field(shape, K, noise, seed)
    ids = oracle.authorized_by_persistence(f, 0.05)
    g, O = oracle.lts(f, ids, mode="both")
    return (i, W.sha256_of(g), W.sha256_of(O))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs, _ = _specs()
    sizes = [int(np.prod(s[0])) for s in specs]
    res = S.run_sharded(sizes, _simplify_one, rank, world, dist)
    out[rank] = (res, S.shard_fields(sizes, world)[rank])
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_simplify_their_shares_and_gather_the_single_process_results():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    specs, _ = _specs()
    single = [_simplify_one(i) for i in range(len(specs))]
    assert out[0][0] == single and out[1][0] == single
    assert sorted(out[0][1] + out[1][1]) == list(range(len(specs)))
    assert set(out[0][1]).isdisjoint(out[1][1])


def _bench_rank(rank, world, port, out):
    """bench.py's rank helper on gloo: the slowest rank's time, summed rates, gathered objects."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    r = bench._Ranks(dist, rank, world, torch.device("cpu"))
    out[rank] = (r.reduce([1.5, 4.0][rank], "max"), r.reduce([10.0, 32.0][rank], "sum"),
                 r.reduce([1.0, 0.0][rank], "min"), r.gather((rank, [rank] * (rank + 1))))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_rank_helpers_on_two_gloo_ranks():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_bench_rank, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1]
    mx, sm, mn, gathered = out[0]
    assert (mx, sm, mn) == (4.0, 42.0, 0.0)
    assert gathered == [(0, [0]), (1, [1, 1])]
