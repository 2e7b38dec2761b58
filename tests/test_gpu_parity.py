"""Parity of the CUDA library (through its C ABI) with the oracle.

The method is integer and copy work, so the bar is bit-exact equality of the
simplified field g (compared as raw bits) and of the order field, on the same
seeded inputs."""
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


def run_gpu(ctx, f, ids, mode="both"):
    dev = torch.device("cuda", 0)
    g, o, st = ctx.simplify(torch.from_numpy(np.ascontiguousarray(f)).to(dev),
                            torch.from_numpy(np.ascontiguousarray(ids, dtype=np.int32)).to(dev), mode)
    torch.cuda.synchronize()
    return g.cpu().numpy(), o.cpu().numpy(), st


def assert_same(g, o, g_ref, o_ref, what=""):
    assert np.array_equal(o, o_ref), f"order field differs {what}: {int(np.sum(o != o_ref))} vertices"
    assert np.array_equal(g.view(np.uint32), g_ref.view(np.uint32)), \
        f"field differs {what}: {int(np.sum(g.view(np.uint32) != g_ref.view(np.uint32)))} vertices"


def random_ids(rng, f, p):
    O = oracle.order_field(f).reshape(-1)
    ids = np.nonzero(rng.random(f.size) < p)[0]
    return np.concatenate([ids, [np.argmax(O), np.argmin(O)]]).astype(np.int32)


@pytest.mark.parametrize("mode", ["min", "max", "both"])
def test_tiny_random_grids(ctx_small, mode):
    rng = np.random.default_rng({"min": 1, "max": 2, "both": 3}[mode])
    for it in range(40):
        dim3 = it % 2 == 1
        shape = tuple(int(rng.integers(2, 7 if dim3 else 13)) for _ in range(3 if dim3 else 2))
        f = W.random_tiny_field(rng, shape, levels=None if it % 3 else 5)
        ids = random_ids(rng, f, 0.1)
        g_ref, o_ref = oracle.lts(f, ids, mode=mode)
        g, o, _ = run_gpu(ctx_small, f, ids, mode)
        assert_same(g, o, g_ref, o_ref, f"{shape} it={it}")


def test_ragged_and_thin_grids(ctx_small):
    rng = np.random.default_rng(17)
    for shape in [(2, 2), (2, 3), (3, 2), (2, 2, 2), (2, 1000), (1001, 2), (3, 2, 517), (33, 65), (5, 7, 131)]:
        f = W.random_tiny_field(rng, shape, levels=7)
        ids = random_ids(rng, f, 0.05)
        g_ref, o_ref = oracle.lts(f, ids, mode="both")
        g, o, _ = run_gpu(ctx_small, f, ids)
        assert_same(g, o, g_ref, o_ref, str(shape))


def test_order_field_only_parity(ctx_small):
    """All extrema authorized: nothing moves, the output is (f, order field of f)."""
    rng = np.random.default_rng(5)
    for shape in [(64, 48), (17, 23, 29), (4097, 3)]:
        f = W.random_tiny_field(rng, shape, levels=11)
        f[0, 0] = -0.0
        f.reshape(-1)[5] = 0.0
        O = oracle.order_field(f)
        nbr = H.neighbour_table(shape) if f.size < 30000 else None
        if nbr is not None:
            mins, maxs = H.extrema(O, nbr)
            ids = np.array(sorted(mins | maxs), np.int32)
        else:
            ids = np.arange(f.size, dtype=np.int32)
        g, o, st = run_gpu(ctx_small, f, ids)
        assert np.array_equal(o, O)
        assert np.array_equal(g.view(np.uint32), f.view(np.uint32))
        assert st["removed"] == [0, 0]


@pytest.mark.parametrize("config", [0, 1])
def test_gaussian_configs(lts, config):
    f = W.make_config_field(config)
    ids = oracle.authorized_by_persistence(f, W.CONFIGS[config]["thr"])
    g_ref, o_ref, st_ref = oracle.lts(f, ids, mode="both", return_stats=True)
    ctx = lts.Context(f.size, device=0)
    g, o, st = run_gpu(ctx, f, ids)
    ctx.close()
    assert_same(g, o, g_ref, o_ref, f"config {config}")
    assert st["removed"] == [st_ref["removed_min"], st_ref["removed_max"]]
    assert st["regions"] == [st_ref["regions_min"], st_ref["regions_max"]]
    assert st["region_vertices"] == [st_ref["region_vertices_min"], st_ref["region_vertices_max"]]
    assert st["max_local_floods"] == [st_ref["max_local_floods_min"], st_ref["max_local_floods_max"]]
    assert st["fallback_regions"] == [st_ref["fallback_regions_min"], st_ref["fallback_regions_max"]]


@pytest.mark.parametrize("side", [64, 128])
def test_boxnoise_small(lts, side):
    f = W.make_config_field(2, shape=(side, side, side))
    ids = oracle.authorized_by_persistence(f, W.CONFIGS[2]["thr"])
    g_ref, o_ref = oracle.lts(f, ids, mode="both")
    ctx = lts.Context(f.size, device=0)
    g, o, st = run_gpu(ctx, f, ids)
    ctx.close()
    assert_same(g, o, g_ref, o_ref, f"box noise {side}^3")


def test_random_authorized_sets_and_repeat(ctx_small):
    """Arbitrary authorized sets (not persistence-based), repeated calls on one context."""
    rng = np.random.default_rng(23)
    f = W.make_config_field(0, shape=(96, 80))
    for it in range(4):
        ids = random_ids(rng, f, 0.02 * (it + 1))
        g_ref, o_ref = oracle.lts(f, ids, mode="both")
        for rep in range(2):
            g, o, _ = run_gpu(ctx_small, f, ids)
            assert_same(g, o, g_ref, o_ref, f"it={it} rep={rep}")


def _golden(name):
    from tests.golden import store as mg

    if not os.path.exists(os.path.join(GOLDEN, f"{name}.json")):
        pytest.skip(f"no stored values for {name}")
    return mg.load_record(name), mg.load_authorized(name)


@pytest.mark.parametrize("name", ["boxnoise3d_256", "boxnoise3d_512"])
def test_boxnoise_full_size_against_stored_oracle_hashes(lts, name):
    rec, ids = _golden(name)
    cfg = rec["config"]
    shape = tuple(rec["shape"])
    f = W.make_config_field(cfg, shape=shape)
    assert W.sha256_of(f) == rec["field_sha256"], "generator output differs from the stored field"
    assert ids.size == rec["n_authorized"]
    ctx = lts.Context(f.size, device=0)
    g, o, st = run_gpu(ctx, f, ids)
    ctx.close()
    s = rec["stats"]
    assert st["removed"] == [s["removed_min"], s["removed_max"]]
    assert st["regions"] == [s["regions_min"], s["regions_max"]]
    assert st["region_vertices"] == [s["region_vertices_min"], s["region_vertices_max"]]
    assert W.sha256_of(o) == rec["order_sha256"]
    assert W.sha256_of(g) == rec["g_sha256"]


# ---------------------------------------------------------------------------
# errors reported through the ABI
# ---------------------------------------------------------------------------

def test_errors(lts, ctx_small):
    dev = torch.device("cuda", 0)
    f = W.make_config_field(0, shape=(32, 32))
    ids = oracle.authorized_by_persistence(f, 0.05)
    # NaN in the field
    fn = f.copy()
    fn[3, 4] = np.nan
    with pytest.raises(lts.LtsError) as e:
        run_gpu(ctx_small, fn, ids)
    assert e.value.code == 2
    # authorized id out of range
    with pytest.raises(lts.LtsError) as e:
        run_gpu(ctx_small, f, np.array([f.size + 5], np.int32))
    assert e.value.code == 1
    # no authorized maximum while maxima must be removed
    O = oracle.order_field(f).reshape(-1)
    with pytest.raises(lts.LtsError) as e:
        run_gpu(ctx_small, f, np.array([int(np.argmin(O))], np.int32), "max")
    assert e.value.code == 3
    # output aliasing the input
    ft = torch.from_numpy(f).to(dev)
    it = torch.from_numpy(ids).to(dev)
    with pytest.raises(lts.LtsError) as e:
        ctx_small.simplify(ft, it, "both", out_field=ft)
    assert e.value.code == 1
    # the context still works after errors
    g_ref, o_ref = oracle.lts(f, ids, mode="both")
    g, o, _ = run_gpu(ctx_small, f, ids)
    assert_same(g, o, g_ref, o_ref, "after errors")


# ---------------------------------------------------------------------------
# the order field's two sorts (few distinct values: two digit passes on
# compressed keys; otherwise four) and pointers that are not 16-byte aligned
# ---------------------------------------------------------------------------

def order_by_simplify(lts, ctx, f):
    """lts_simplify with every vertex authorized returns (f, order field of f)."""
    dev = torch.device("cuda", 0)
    g, o, st = ctx.simplify(torch.from_numpy(np.ascontiguousarray(f)).to(dev),
                            torch.arange(f.size, dtype=torch.int32, device=dev), "both")
    torch.cuda.synchronize()
    assert st["removed"] == [0, 0]
    return o.cpu().numpy()


@pytest.mark.parametrize("distinct", [1, 2, 255, 256, 4095, 4096, 4097, 9000])
def test_order_field_around_the_distinct_key_threshold(lts, ctx_small, distinct):
    rng = np.random.default_rng(1000 + distinct)
    shape = (96, 150)                       # 14,400 vertices, several tiles and a ragged tail
    vals = np.arange(shape[0] * shape[1]) % distinct
    vals = rng.permutation(vals).astype(np.float32) * np.float32(0.37) - np.float32(700.0)
    f = vals.reshape(shape)
    if distinct in (255, 9000):
        f.reshape(-1)[:3] = [-0.0, 0.0, np.inf]   # -0 == +0 (one key), infinities are keys too
    o = order_by_simplify(lts, ctx_small, f)
    assert np.array_equal(o, oracle.order_field(f))


def test_unaligned_input_and_output_pointers(lts, ctx_small):
    """Views one float into larger buffers: the histogram pass takes its
    scalar path for every chunk."""
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(31)
    for shape, levels in [((61, 77), 9), ((13, 17, 19), None)]:
        f = W.random_tiny_field(rng, shape, levels)
        ids = random_ids(rng, f, 0.1)
        g_ref, o_ref = oracle.lts(f, ids, mode="both")
        n = f.size
        fb = torch.zeros(n + 1, dtype=torch.float32, device=dev)
        fb[1:] = torch.from_numpy(f.reshape(-1)).to(dev)
        gb = torch.empty(n + 1, dtype=torch.float32, device=dev)
        ob = torch.empty(n + 1, dtype=torch.int32, device=dev)
        fv, gv, ov = fb[1:].view(shape), gb[1:].view(shape), ob[1:].view(shape)
        assert fv.data_ptr() % 16 != 0 and gv.data_ptr() % 16 != 0
        idd = torch.from_numpy(ids).to(dev)
        code = lts.lts_simplify(ctx_small._ctx, lts.grid_of_shape(shape), fv.data_ptr(), idd.data_ptr(), idd.numel(),
                                "both", gv.data_ptr(), ov.data_ptr())
        assert code == 0, lts.lts_last_error(ctx_small._ctx)
        torch.cuda.synchronize()
        assert_same(gv.cpu().numpy(), ov.cpu().numpy(), g_ref, o_ref, f"unaligned {shape}")
