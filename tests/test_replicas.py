"""The multi-rank path of bench.py (one replica per rank, no collective on
the data path): the per-step time is the slowest rank's and the value counts
every rank's vertices.  Two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [12.5, 20.0][rank]
    ms = bench.slowest_rank_ms(local_ms, dist, torch.device("cpu"))
    out[rank] = (ms, bench.whole_job_mvps(1000000, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_all_vertices():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == 20.0
    assert value == pytest.approx(2 * 1000000 / 0.020 / 1e6)


def test_single_rank_is_local():
    import bench

    assert bench.slowest_rank_ms(7.0, None, None) == 7.0
    assert bench.whole_job_mvps(134217728, 1, 33.9) == pytest.approx(134217728 / 0.0339 / 1e6)
