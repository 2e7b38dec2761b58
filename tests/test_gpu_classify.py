"""lts_classify (Sec. 3.1 critical points from the link lookup table) against
the oracle's brute-force link classification, per vertex, on random orders,
the output of a simplification, and textbook saddles; counts from the
per-vertex values."""
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


def _classify(lts, ctx, O):
    dev = torch.device("cuda", 0)
    od = torch.from_numpy(np.ascontiguousarray(O, dtype=np.int32)).to(dev)
    lo = torch.empty(O.shape, dtype=torch.int8, device=dev)
    up = torch.empty(O.shape, dtype=torch.int8, device=dev)
    code, counts = lts.lts_classify(ctx._ctx, lts.grid_of_shape(O.shape), od.data_ptr(), lo.data_ptr(), up.data_ptr())
    assert code == 0, lts.lts_last_error(ctx._ctx)
    torch.cuda.synchronize()
    return lo.cpu().numpy(), up.cpu().numpy(), counts


def _expected_counts(lo, up):
    lo = lo.astype(np.int64).reshape(-1)
    up = up.astype(np.int64).reshape(-1)
    mn = int(np.sum(lo == 0))
    mx = int(np.sum((up == 0) & (lo != 0)))
    reg = int(np.sum((lo == 1) & (up == 1)))
    return [mn, mx, reg, lo.size - mn - mx - reg, int(np.sum(np.maximum(lo - 1, 0))), int(np.sum(np.maximum(up - 1, 0)))]


@pytest.mark.parametrize("shape", [(2, 2), (7, 9), (64, 80), (3, 4, 5), (17, 23, 29), (2, 2, 2), (64, 64, 64)])
def test_random_orders_match_the_oracle(lts, ctx, shape):
    rng = np.random.default_rng(int(np.prod(shape)))
    O = rng.permutation(int(np.prod(shape))).astype(np.int32).reshape(shape)
    lo, up, counts = _classify(lts, ctx, O)
    lo_ref, up_ref = oracle.classify(O)
    assert np.array_equal(lo, lo_ref) and np.array_equal(up, up_ref)
    assert counts == _expected_counts(lo_ref, up_ref)


def test_simplified_output_has_only_authorized_extrema(lts, ctx):
    f = W.make_config_field(1, shape=(96, 96, 96))
    ids = oracle.authorized_by_persistence(f, W.CONFIGS[1]["thr"])
    dev = torch.device("cuda", 0)
    g, o, st = ctx.simplify(torch.from_numpy(f).to(dev), torch.from_numpy(ids).to(dev), "both")
    torch.cuda.synchronize()
    O = o.cpu().numpy()
    lo, up, counts = _classify(lts, ctx, O)
    lo_ref, up_ref = oracle.classify(O)
    assert np.array_equal(lo, lo_ref) and np.array_equal(up, up_ref)
    ext = set(np.nonzero((lo.reshape(-1) == 0) | (up.reshape(-1) == 0))[0].tolist())
    assert ext == set(ids.tolist()) & ext and counts[0] + counts[1] == len(ext)
    assert ext <= set(ids.tolist())                        # Eq. 1 on the GPU's own output


