"""lts_order_field_static (the order field computed on the library's static
scratch, with no allocation at call time) against the existing entry point:
lts_simplify with every vertex authorized returns the order field of its
input unchanged.  Both are called through the C ABI; each case calls the
static entry point twice in a row, so a result that depends on scratch left
over from an earlier call shows up.  The file is collected last so that it
also runs after every other GPU test in the same process."""
import zlib

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


def order_by_simplify(lts, f_dev, stream):
    """The existing path: lts_simplify with all ids authorized -> (g, O) = (f, order field)."""
    n = f_dev.numel()
    ctx = lts.lts_create(0, n, stream.cuda_stream)
    try:
        ids = torch.arange(n, dtype=torch.int32, device=f_dev.device)
        g = torch.empty_like(f_dev)
        o = torch.full(f_dev.shape, -1, dtype=torch.int32, device=f_dev.device)
        torch.cuda.synchronize()
        code = lts.lts_simplify(ctx, lts.grid_of_shape(tuple(f_dev.shape)), f_dev.data_ptr(), ids.data_ptr(), n,
                                "both", g.data_ptr(), o.data_ptr())
        assert code == 0, lts.lts_last_error(ctx)
        stream.synchronize()
        assert torch.equal(g.view(torch.int32), f_dev.view(torch.int32))
        return o.cpu().numpy()
    finally:
        lts.lts_destroy(ctx)


def order_static(lts, f_dev, stream):
    o = torch.full(f_dev.shape, -1, dtype=torch.int32, device=f_dev.device)
    torch.cuda.synchronize()
    code, msg = lts.lts_order_field_static(0, lts.grid_of_shape(tuple(f_dev.shape)), f_dev.data_ptr(),
                                           o.data_ptr(), stream.cuda_stream)
    assert code == 0, msg
    assert msg == ""
    return o.cpu().numpy()


CASES = [
    ("2d_ragged_ties", (37, 53), 5),
    ("3d_ragged", (17, 23, 29), None),
    ("3d_max_ties", (64, 128, 128), 97),   # exactly LTS_ORDER_STATIC_MAX_VERTICES
    ("2d_tiny", (2, 2), 2),
    ("2d_max", (1024, 1024), None),
    ("3d_one_tile_and_a_bit", (2, 2, 1025), 13),
]


@pytest.mark.parametrize("name,shape,levels", CASES, ids=[c[0] for c in CASES])
def test_static_order_field_matches_lts_simplify_twice(lts, name, shape, levels):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    f = W.random_tiny_field(rng, shape, levels)
    f.reshape(-1)[0] = -0.0
    f.reshape(-1)[-1] = 0.0
    dev = torch.device("cuda", 0)
    f_dev = torch.from_numpy(f).to(dev)
    stream = torch.cuda.current_stream(dev) if len(shape) == 2 else torch.cuda.Stream(dev)
    expect = order_by_simplify(lts, f_dev, stream)
    first = order_static(lts, f_dev, stream)
    second = order_static(lts, f_dev, stream)
    assert np.array_equal(first, expect), f"first call: {int(np.sum(first != expect))} vertices differ"
    assert np.array_equal(second, expect), f"second call: {int(np.sum(second != expect))} vertices differ"
    assert np.array_equal(first, oracle.order_field(f))   # the oracle at every size, 2^20 included
    assert torch.equal(f_dev.cpu().view(torch.int32), torch.from_numpy(f).view(torch.int32))   # input untouched


def test_static_order_field_errors(lts):
    dev = torch.device("cuda", 0)
    f = torch.zeros((1025, 1024), dtype=torch.float32, device=dev)
    o = torch.empty((1025, 1024), dtype=torch.int32, device=dev)
    code, msg = lts.lts_order_field_static(0, lts.grid_of_shape((1025, 1024)), f.data_ptr(), o.data_ptr())
    assert code == 1 and "at most 1048576" in msg
    g = torch.arange(64 * 48, dtype=torch.float32, device=dev).reshape(64, 48)
    g[3, 7] = float("nan")
    o2 = torch.empty((64, 48), dtype=torch.int32, device=dev)
    code, msg = lts.lts_order_field_static(0, lts.grid_of_shape((64, 48)), g.data_ptr(), o2.data_ptr())
    assert code == 2 and "NaN" in msg
    # a failed call leaves nothing behind: the next one is exact
    g[3, 7] = 0.5
    code, msg = lts.lts_order_field_static(0, lts.grid_of_shape((64, 48)), g.data_ptr(), o2.data_ptr())
    assert code == 0, msg
    assert np.array_equal(o2.cpu().numpy(), oracle.order_field(g.cpu().numpy()))
