"""Launch tunings (lts_set_tuning) change no result: plain, persistence-driven
and batched calls under extreme tunings are bit-identical to the defaults'."""
import numpy as np
import pytest

import oracle
from paper_2009_00083_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TUNINGS = [{"engine_blocks_per_sm": 1, "team_blocks_per_sm": 1, "batch_workspaces": 1},
           {"engine_blocks_per_sm": 4, "team_blocks_per_sm": 16, "batch_workspaces": 2},
           {"engine_blocks_per_sm": 6, "team_blocks_per_sm": 8, "batch_workspaces": 7}]


@pytest.fixture(scope="module")
def lts():
    import paper_2009_00083_gb300 as lts_mod

    lts_mod.load()
    return lts_mod


def _bits(g, o):
    return g.view(torch.int32).cpu().numpy(), o.cpu().numpy()


def test_defaults_and_argument_checks(lts):
    ctx = lts.Context(1 << 16, device=0)
    try:
        assert ctx.tuning() == {"engine_blocks_per_sm": 8, "team_blocks_per_sm": 12, "batch_workspaces": 32}
        for bad in ({"engine_blocks_per_sm": 9}, {"team_blocks_per_sm": -1}, {"batch_workspaces": 33}):
            with pytest.raises(lts.LtsError) as e:
                ctx.set_tuning(bad)
            assert e.value.code == 1
        assert ctx.tuning()["engine_blocks_per_sm"] == 8      # a refused tuning changes nothing
        ctx.set_tuning({"engine_blocks_per_sm": 3})
        assert ctx.tuning() == {"engine_blocks_per_sm": 3, "team_blocks_per_sm": 12, "batch_workspaces": 32}
        ctx.set_tuning(None)
        assert ctx.tuning()["engine_blocks_per_sm"] == 8
    finally:
        ctx.close()


def test_tunings_change_no_result(lts):
    dev = torch.device("cuda", 0)
    f = W.gaussian_field((48, 56, 40), 64, 0.02, seed=W.seed_of(1, 5))
    ids = oracle.authorized_by_persistence(f, 0.01)
    g_ref, o_ref = oracle.lts(f, ids, "both")
    fd, idd = torch.from_numpy(f).to(dev), torch.from_numpy(ids).to(dev)
    eps = 0.01 * float(f.max() - f.min())
    ctx = lts.Context(f.size, device=0)
    try:
        gp0, op0 = _bits(*ctx.simplify_persistence(fd, eps, "both", with_stats=False)[:2])
        for t in TUNINGS:
            ctx.set_tuning(t)
            g, o = _bits(*ctx.simplify(fd, idd, "both", with_stats=False)[:2])
            assert np.array_equal(o, o_ref) and np.array_equal(g, g_ref.view(np.int32)), t
            gp, op = _bits(*ctx.simplify_persistence(fd, eps, "both", with_stats=False)[:2])
            assert np.array_equal(op, op0) and np.array_equal(gp, gp0), t
    finally:
        ctx.close()


def test_batch_workspaces_change_no_result(lts):
    dev = torch.device("cuda", 0)
    cases = []
    for k in range(9):
        shape = (40 + 8 * k, 56) if k % 2 else (20 + k, 24, 18)
        f = W.gaussian_field(shape, 16, 0.05, seed=W.seed_of(3, 100 + k))
        ids = oracle.authorized_by_persistence(f, 0.03)
        cases.append((f, ids) + oracle.lts(f, ids, "both"))
    fields = [torch.from_numpy(c[0]).to(dev) for c in cases]
    auth = [torch.from_numpy(c[1]).to(dev) for c in cases]
    ctx = lts.Context(max(f.numel() for f in fields), device=0)
    try:
        for t in TUNINGS:
            ctx.set_tuning(t)
            outs, _ = ctx.simplify_batch(fields, auth, "both", with_stats=False)
            for (g, o), c in zip(outs, cases):
                gb, ob = _bits(g, o)
                assert np.array_equal(ob, c[3]) and np.array_equal(gb, c[2].view(np.int32)), t
    finally:
        ctx.close()
