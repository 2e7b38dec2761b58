"""lts_simplify_f64 (a float64 field) through the C ABI against the oracle's
float64 path, bit for bit: order field and simplified field."""
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


@pytest.fixture(scope="module")
def ctx(lts):
    c = lts.Context(1 << 21, device=0)
    yield c
    c.close()


def _gpu(ctx, f, ids, mode="both"):
    dev = torch.device("cuda", 0)
    g, o, st = ctx.simplify(torch.from_numpy(np.ascontiguousarray(f)).to(dev),
                            torch.from_numpy(np.ascontiguousarray(ids, dtype=np.int32)).to(dev), mode)
    torch.cuda.synchronize()
    return g.cpu().numpy(), o.cpu().numpy(), st


def _same(g, o, g_ref, o_ref, what):
    assert g.dtype == np.float64
    assert np.array_equal(o, o_ref), f"{what}: order differs at {int(np.sum(o != o_ref))} vertices"
    assert np.array_equal(g.view(np.uint64), g_ref.view(np.uint64)), f"{what}: field differs"


def _ids(rng, O, p):
    O = O.reshape(-1)
    return np.concatenate([np.nonzero(rng.random(O.size) < p)[0], [np.argmax(O), np.argmin(O)]]).astype(np.int32)


@pytest.mark.parametrize("mode", ["min", "max", "both"])
def test_tiny_random_float64_grids(ctx, mode):
    rng = np.random.default_rng({"min": 4, "max": 5, "both": 6}[mode])
    for it in range(30):
        dim3 = it % 2 == 1
        shape = tuple(int(rng.integers(2, 7 if dim3 else 14)) for _ in range(3 if dim3 else 2))
        f = rng.normal(size=shape)
        if it % 3 == 0:
            f = np.round(f, 1)                                   # ties
        f.reshape(-1)[0] = -0.0
        if f.size > 3:
            f.reshape(-1)[1] = 0.0
            f.reshape(-1)[2] = np.inf
        ids = _ids(rng, oracle.order_field_f64(f), 0.1)
        g_ref, o_ref = oracle.lts_f64(f, ids, mode)
        g, o, _ = _gpu(ctx, f, ids, mode)
        _same(g, o, g_ref, o_ref, f"{shape} it={it}")


def test_ties_that_exist_only_in_float32(ctx):
    shape = (48, 64)
    rng = np.random.default_rng(8)
    k = rng.permutation(shape[0] * shape[1]).reshape(shape)
    f = 1.0 + k.astype(np.float64) * 2.0 ** -40
    ids = _ids(rng, oracle.order_field_f64(f), 0.02)
    g_ref, o_ref = oracle.lts_f64(f, ids)
    g, o, _ = _gpu(ctx, f, ids)
    _same(g, o, g_ref, o_ref, "float64-only values")
    assert not np.array_equal(oracle.order_field_f64(f), oracle.order_field(f.astype(np.float32)))


@pytest.mark.parametrize("which", ["config0", "config1_64", "boxnoise_64"])
def test_float64_workloads(ctx, which):
    if which == "config0":
        f = W.gaussian_field((256, 256), 16, 0.05, W.seed_of(0), dtype=np.float64)
        thr = W.CONFIGS[0]["thr"]
    elif which == "config1_64":
        f = W.gaussian_field((64, 64, 64), 64, 0.02, W.seed_of(1), dtype=np.float64)
        thr = W.CONFIGS[1]["thr"]
    else:
        f = W.make_config_field(2, shape=(64, 64, 64)).astype(np.float64)
        thr = W.CONFIGS[2]["thr"]
    # persistence-selected extrema: the float32 selector on the rounded field
    # authorizes ids; the float64 method uses them as a plain list
    ids = oracle.authorized_by_persistence(f.astype(np.float32), thr)
    O64 = oracle.order_field_f64(f).reshape(-1)
    ids = np.unique(np.concatenate([ids, [np.argmax(O64), np.argmin(O64)]])).astype(np.int32)
    g_ref, o_ref, st_ref = oracle.lts_f64(f, ids, return_stats=True)
    g, o, st = _gpu(ctx, f, ids)
    _same(g, o, g_ref, o_ref, which)
    assert st["removed"] == [st_ref["removed_min"], st_ref["removed_max"]]


def test_float64_equals_float32_on_float32_values(ctx):
    f32 = W.make_config_field(2, shape=(48, 40, 44))
    ids = oracle.authorized_by_persistence(f32, 0.1)
    dev = torch.device("cuda", 0)
    a, b, _ = ctx.simplify(torch.from_numpy(f32).to(dev), torch.from_numpy(ids).to(dev), "both")
    c, d, _ = ctx.simplify(torch.from_numpy(f32.astype(np.float64)).to(dev), torch.from_numpy(ids).to(dev), "both")
    torch.cuda.synchronize()
    assert torch.equal(b, d)
    assert torch.equal(a.double(), c)


def test_float64_errors(lts, ctx):
    dev = torch.device("cuda", 0)
    f = torch.zeros((32, 40), dtype=torch.float64, device=dev)
    f[3, 4] = float("nan")
    ids = torch.tensor([0], dtype=torch.int32, device=dev)
    with pytest.raises(lts.LtsError) as e:
        ctx.simplify(f, ids, "both")
    assert e.value.code == 2
    # an output that overlaps the input's second half (8 bytes per vertex)
    f[3, 4] = 0.5
    buf = torch.zeros(2 * 32 * 40, dtype=torch.float64, device=dev)
    buf[: 32 * 40] = f.reshape(-1)
    o = torch.empty((32, 40), dtype=torch.int32, device=dev)
    code = lts.lts_simplify_f64(ctx._ctx, lts.grid_of_shape((32, 40)), buf.data_ptr(), ids.data_ptr(), 1, "both",
                                buf.data_ptr() + 8 * 32 * 20, o.data_ptr())
    assert code == 1
    # the context is fine afterwards
    fh = f.cpu().numpy()
    Oh = oracle.order_field_f64(fh).reshape(-1)
    keep = np.array([np.argmin(Oh), np.argmax(Oh)], np.int32)
    g, o2, _ = ctx.simplify(f, torch.from_numpy(keep).to(dev), "both")
    torch.cuda.synchronize()
    assert np.array_equal(o2.cpu().numpy(), oracle.lts_f64(fh, keep)[1])
