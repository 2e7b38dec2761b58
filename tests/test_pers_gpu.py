"""Parity of persistence-driven LTS (Sec. 4.5) through the C ABI
(lts_simplify_persistence) with the oracle's pers_lts (Elder-rule selection
per pass, then the pass): bit-exact simplified field (raw bits) and order
field on the same seeded inputs, and the same counts of removed extrema."""
import os

import numpy as np
import pytest

import oracle
from paper_2009_00083_gb300 import workloads as W
from tests import helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def lts():
    import paper_2009_00083_gb300 as lts_mod

    lts_mod.load()
    return lts_mod


@pytest.fixture(scope="module")
def ctx_small(lts):
    c = lts.Context(1 << 22, device=0)
    yield c
    c.close()


def run_pers(ctx, f, eps, mode="both"):
    dev = torch.device("cuda", 0)
    g, o, st = ctx.simplify_persistence(torch.from_numpy(np.ascontiguousarray(f)).to(dev), eps, mode)
    torch.cuda.synchronize()
    return g.cpu().numpy(), o.cpu().numpy(), st


def assert_same(g, o, g_ref, o_ref, what=""):
    assert np.array_equal(o, o_ref), f"order field differs {what}: {int(np.sum(o != o_ref))} vertices"
    assert np.array_equal(g.view(np.uint32), g_ref.view(np.uint32)), \
        f"field differs {what}: {int(np.sum(g.view(np.uint32) != g_ref.view(np.uint32)))} vertices"


def frange(f):
    return float(np.float64(f.max()) - np.float64(f.min()))


def eps_choices(f, rng):
    """0, exact persistence values of f (p == eps is not kept), a fraction of the range, beyond the range."""
    pmin, pmax = oracle.persistence(f)
    p = np.concatenate([pmin[~np.isnan(pmin)], pmax[~np.isnan(pmax)]])
    return [0.0, float(rng.choice(p)), float(rng.choice(p)), 0.2 * frange(f), 3.0 * frange(f) + 1.0]


@pytest.mark.parametrize("mode", ["min", "max", "both"])
def test_tiny_random_grids(ctx_small, mode):
    rng = np.random.default_rng({"min": 71, "max": 72, "both": 73}[mode])
    for it in range(24):
        dim3 = it % 2 == 1
        shape = tuple(int(rng.integers(2, 7 if dim3 else 13)) for _ in range(3 if dim3 else 2))
        f = W.random_tiny_field(rng, shape, levels=None if it % 3 else 5)
        for eps in eps_choices(f, rng):
            g_ref, o_ref = oracle.pers_lts(f, eps, mode=mode)
            g, o, _ = run_pers(ctx_small, f, eps, mode)
            assert_same(g, o, g_ref, o_ref, f"{shape} it={it} eps={eps}")


def test_ragged_and_thin_grids(ctx_small):
    rng = np.random.default_rng(77)
    for shape in [(2, 2), (2, 3), (3, 2), (2, 2, 2), (2, 1000), (1001, 2), (3, 2, 517), (33, 65), (5, 7, 131)]:
        f = W.random_tiny_field(rng, shape, levels=7)
        eps = 0.3 * frange(f)
        g_ref, o_ref = oracle.pers_lts(f, eps, mode="both")
        g, o, _ = run_pers(ctx_small, f, eps)
        assert_same(g, o, g_ref, o_ref, str(shape))


@pytest.mark.parametrize("config", [0, 1])
def test_gaussian_configs(lts, config):
    f = W.make_config_field(config)
    eps = W.CONFIGS[config]["thr"] * frange(f)
    g_ref, o_ref = oracle.pers_lts(f, eps, mode="both")
    ctx = lts.Context(f.size, device=0)
    g, o, st = run_pers(ctx, f, eps)
    ctx.close()
    assert_same(g, o, g_ref, o_ref, f"config {config}")
    assert np.max(np.abs(g.astype(np.float64) - f)) <= eps


@pytest.mark.parametrize("side,thr", [(64, 0.10), (128, 0.10), (96, 0.02)])
def test_boxnoise_small(lts, side, thr):
    f = W.make_config_field(2, shape=(side, side, side))
    eps = thr * frange(f)
    g_ref, o_ref = oracle.pers_lts(f, eps, mode="both")
    ctx = lts.Context(f.size, device=0)
    g, o, _ = run_pers(ctx, f, eps)
    ctx.close()
    assert_same(g, o, g_ref, o_ref, f"box noise {side}^3 thr {thr}")


@pytest.mark.parametrize("mode", ["min", "max"])
def test_single_pass_equals_lts_with_the_elder_rule_selection(lts, mode):
    """One pass of Pers-LTS equals LTS with the extrema selected by persistence on f."""
    f = W.make_config_field(1)
    thr = W.CONFIGS[1]["thr"]
    ids = oracle.authorized_by_persistence(f, thr)
    g_ref, o_ref, st_ref = oracle.lts(f, ids, mode=mode, return_stats=True)
    ctx = lts.Context(f.size, device=0)
    g, o, st = run_pers(ctx, f, thr * frange(f), mode)
    ctx.close()
    assert_same(g, o, g_ref, o_ref, mode)
    side = 0 if mode == "min" else 1
    assert st["removed"][side] == st_ref["removed_" + mode]
    assert st["regions"][side] == st_ref["regions_" + mode]


def test_interleaved_with_lists_and_repeated(ctx_small):
    """Persistence-driven and list-driven calls alternate on one context."""
    rng = np.random.default_rng(79)
    f = W.make_config_field(0, shape=(150, 130))
    dev = torch.device("cuda", 0)
    for it in range(3):
        eps = (0.01 + 0.04 * it) * frange(f)
        g_ref, o_ref = oracle.pers_lts(f, eps, mode="both")
        for rep in range(2):
            g, o, _ = run_pers(ctx_small, f, eps)
            assert_same(g, o, g_ref, o_ref, f"it={it} rep={rep}")
        ids = oracle.authorized_by_persistence(f, 0.03)
        g2_ref, o2_ref = oracle.lts(f, ids, mode="both")
        g2, o2, _ = ctx_small.simplify(torch.from_numpy(f).to(dev), torch.from_numpy(ids).to(dev), "both")
        assert_same(g2.cpu().numpy(), o2.cpu().numpy(), g2_ref, o2_ref, f"list call after it={it}")


def test_persistent_extrema_are_what_remains(ctx_small):
    f = W.make_config_field(0, shape=(120, 100))
    eps = 0.05 * frange(f)
    g, o, st = run_pers(ctx_small, f, eps, "max")
    nbr = H.neighbour_table(f.shape)
    O = oracle.order_field(f)
    maxs_f = H.extrema(O, nbr)[1]
    maxs_g = H.extrema(o, nbr)[1]
    assert maxs_g == set(oracle.persistent_by_elder(f, O, 1, eps).tolist())
    assert st["removed"][1] == len(maxs_f) - len(maxs_g)


def _golden_pers(name):
    from tests.golden import store

    if not os.path.exists(os.path.join(GOLDEN, f"{name}_pers.json")):
        pytest.skip(f"no stored values for {name}")
    return store.load_record(f"{name}_pers")


@pytest.mark.parametrize("name", ["boxnoise3d_256", "boxnoise3d_512"])
def test_boxnoise_full_size_against_stored_oracle_hashes(lts, name):
    rec = _golden_pers(name)
    f = W.make_config_field(rec["config"], shape=tuple(rec["shape"]))
    assert W.sha256_of(f) == rec["field_sha256"], "generator output differs from the stored field"
    eps = rec["thr"] * frange(f)
    assert eps == rec["eps"]
    ctx = lts.Context(f.size, device=0)
    g, o, st = run_pers(ctx, f, eps)
    ctx.close()
    assert W.sha256_of(o) == rec["order_sha256"]
    assert W.sha256_of(g) == rec["g_sha256"]
    assert float(np.max(np.abs(g.astype(np.float64) - f))) == rec["max_abs_change"] <= eps


def test_errors(lts, ctx_small):
    f = W.make_config_field(0, shape=(40, 30))
    for bad in (-1.0, float("nan"), -0.5e-30):
        with pytest.raises(lts.LtsError) as e:
            run_pers(ctx_small, f, bad)
        assert e.value.code == 1
    fn = f.copy()
    fn[3, 4] = np.nan
    with pytest.raises(lts.LtsError) as e:
        run_pers(ctx_small, fn, 0.1)
    assert e.value.code == 2
    # infinities are ordered like any value; eps = inf keeps only the global extrema
    fi = f.copy()
    fi[10, 10] = np.inf
    fi[20, 5] = -np.inf
    for eps in (0.05 * frange(f), float("inf")):
        g_ref, o_ref = oracle.pers_lts(fi, eps)
        g, o, _ = run_pers(ctx_small, fi, eps)
        assert_same(g, o, g_ref, o_ref, f"infinities eps={eps}")
    # the context still works after errors
    eps = 0.05 * frange(f)
    g_ref, o_ref = oracle.pers_lts(f, eps)
    g, o, _ = run_pers(ctx_small, f, eps)
    assert_same(g, o, g_ref, o_ref, "after errors")
