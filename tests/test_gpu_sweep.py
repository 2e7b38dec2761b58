"""The output-sensitivity sweep of Fig. 6 (Sec. 5) on the GPU, against the oracle.

Uniform white noise with a random share p of the extrema removed (every
vertex authorized but a random p% of them, never the global minimum or
maximum).  At p = 100 only the global extrema stay and the regions cover a
large share of the grid: at 256^3 the propagations' queues outgrow the flood
overflow-heap pool a workspace starts with, so the call enlarges the pool and
runs again."""
import numpy as np
import pytest

import oracle
from paper_2009_00083_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lts():
    import paper_2009_00083_gb300 as lts_mod

    lts_mod.load()
    return lts_mod


def _run(lts, ctx, f, ids):
    dev = torch.device("cuda", 0)
    g, o, st = ctx.simplify(torch.from_numpy(f).to(dev), torch.from_numpy(ids).to(dev), "both")
    torch.cuda.synchronize()
    return g.cpu().numpy(), o.cpu().numpy(), st


@pytest.mark.parametrize("side", [64, 128])
def test_sweep_points_against_the_oracle(lts, side):
    f = W.uniform_noise_field((side,) * 3, W.seed_of(5))
    pts = (0, 50, 90, 99, 100) if side == 64 else (99, 100)
    lists = W.sweep_authorized(f, pts, W.seed_of(5, 1))
    ctx = lts.Context(f.size, device=0)
    try:
        for p, ids in zip(pts, lists):
            g_ref, o_ref, st_ref = oracle.lts(f, ids, "both", return_stats=True)
            g, o, st = _run(lts, ctx, f, ids)
            assert np.array_equal(o, o_ref), f"{side}^3 at {p}%: order differs at {int(np.sum(o != o_ref))} vertices"
            assert np.array_equal(g.view(np.uint32), g_ref.view(np.uint32)), f"{side}^3 at {p}%: field differs"
            assert st["removed"] == [st_ref["removed_min"], st_ref["removed_max"]]
            assert st["max_region"] == [st_ref["max_region_min"], st_ref["max_region_max"]]
    finally:
        ctx.close()


def test_sweep_256_against_stored_oracle_hashes(lts):
    from tests.golden import store

    rec = store.load_record("sweep_256")
    f = W.uniform_noise_field(tuple(rec["shape"]), W.seed_of(5))
    assert W.sha256_of(f) == rec["field_sha256"]
    pts = [p["removed_pct"] for p in rec["points"]]
    lists = W.sweep_authorized(f, pts, W.seed_of(5, 1))
    ctx = lts.Context(f.size, device=0)
    try:
        for pr, ids in zip(rec["points"], lists):
            assert ids.size == pr["n_authorized"]
            g, o, st = _run(lts, ctx, f, ids)
            s = pr["stats"]
            assert st["regions"] == [s["regions_min"], s["regions_max"]], pr["removed_pct"]
            assert W.sha256_of(o) == pr["order_sha256"], pr["removed_pct"]
            assert W.sha256_of(g) == pr["g_sha256"], pr["removed_pct"]
    finally:
        ctx.close()
