"""The optional restoration of swallowed authorized extrema (LTS_MODE_RESTORE,
Sec. 4.2 step 3) on the GPU against the oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2009_00083_gb300 import workloads as W
from tests import helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lts():
    import paper_2009_00083_gb300 as lts_mod

    lts_mod.load()
    return lts_mod


@pytest.fixture(scope="module")
def ctx(lts):
    c = lts.Context(1 << 20, device=0)
    yield c
    c.close()


def _gpu(ctx, f, ids, mode):
    dev = torch.device("cuda", 0)
    g, o, st = ctx.simplify(torch.from_numpy(np.ascontiguousarray(f)).to(dev),
                            torch.from_numpy(np.ascontiguousarray(ids, dtype=np.int32)).to(dev), mode)
    torch.cuda.synchronize()
    return g.cpu().numpy(), o.cpu().numpy(), st


def test_hand_case(ctx):
    f = np.array([[1, 2, 8], [5, 0, 7], [4, 6, 3]], np.float32)
    ids = np.array([2, 4, 6], np.int32)
    g_ref, o_ref = oracle.lts(f, ids, "max+restore")
    g, o, st = _gpu(ctx, f, ids, "max+restore")
    assert np.array_equal(o, o_ref) and np.array_equal(g.view(np.uint32), g_ref.view(np.uint32))
    assert st["restored"] == [0, 1]


@pytest.mark.parametrize("mode", ["min", "max", "both"])
def test_random_arbitrary_authorized_sets(ctx, mode):
    rng = np.random.default_rng({"min": 31, "max": 32, "both": 33}[mode])
    total = 0
    for it in range(150):
        dim3 = it % 3 == 2
        shape = tuple(int(rng.integers(3, 8 if dim3 else 24)) for _ in range(3 if dim3 else 2))
        f = rng.integers(0, 9, size=shape).astype(np.float32) if it % 2 else rng.random(shape).astype(np.float32)
        nbr = H.neighbour_table(shape)
        O = oracle.order_field(f)
        mins, maxs = H.extrema(O, nbr)
        o = O.reshape(-1)
        keep = [v for v in sorted(mins | maxs) if rng.random() < 0.5] + [int(np.argmin(o)), int(np.argmax(o))]
        ids = np.array(sorted(set(keep)), np.int32)
        g_ref, o_ref, st_ref = oracle.lts(f, ids, mode + "+restore", return_stats=True)
        g, oo, st = _gpu(ctx, f, ids, mode + "+restore")
        assert np.array_equal(oo, o_ref), f"{shape} it={it}"
        assert np.array_equal(g.view(np.uint32), g_ref.view(np.uint32))
        assert st["restored"] == [st_ref["restored_min"], st_ref["restored_max"]]
        total += sum(st["restored"])
    assert total > 0


def test_gaussian_field_with_random_authorized_extrema(ctx):
    f = W.gaussian_field((256, 256), 16, 0.05, seed=77)
    nbr = None
    O = oracle.order_field(f)
    rng = np.random.default_rng(3)
    ids = np.nonzero(rng.random(f.size) < 0.3)[0]
    o = O.reshape(-1)
    ids = np.unique(np.concatenate([ids, [np.argmin(o), np.argmax(o)]])).astype(np.int32)
    g_ref, o_ref, st_ref = oracle.lts(f, ids, "both+restore", return_stats=True)
    g, oo, st = _gpu(ctx, f, ids, "both+restore")
    assert np.array_equal(oo, o_ref)
    assert np.array_equal(g.view(np.uint32), g_ref.view(np.uint32))
    assert st["restored"] == [st_ref["restored_min"], st_ref["restored_max"]]
    assert sum(st["restored"]) > 0
