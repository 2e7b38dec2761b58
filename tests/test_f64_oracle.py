"""Pins of the oracle's float64 path (the order field of Sec. 4.1 on float64
values; every later step works on the order field alone).

- The order field equals numpy's lexsort over (value, vertex id) on float64
  data, with -0.0 == +0.0 and infinities ordered, and NaN is rejected.
- On a field whose values are exactly float32 numbers, the float64 method
  gives the float32 method's order field and values (the same ranks, so the
  same regions and local orders, and the same saddle values widened).
- On a field whose float64 values are distinct but collapse to ties in
  float32, the float64 order follows the float64 values (not the float32
  ties broken by id), so the two methods differ exactly where the paper's
  definition says they must.
"""
import numpy as np
import pytest

import oracle
from tests import helpers as H


def _lexsort_rank(f):
    flat = np.asarray(f, dtype=np.float64).reshape(-1).copy()
    flat[flat == 0.0] = 0.0                        # -0.0 and +0.0 are one value
    order = np.lexsort((np.arange(flat.size), flat))
    rank = np.empty(flat.size, dtype=np.int32)
    rank[order] = np.arange(flat.size, dtype=np.int32)
    return rank.reshape(np.shape(f))


@pytest.mark.parametrize("shape", [(7, 9), (5, 6, 7), (33, 3)])
def test_order_field_f64_matches_lexsort(shape):
    rng = np.random.default_rng(sum(shape))
    f = rng.normal(size=shape)
    f.reshape(-1)[::7] = np.round(f.reshape(-1)[::7], 1)        # ties
    f.reshape(-1)[0] = -0.0
    f.reshape(-1)[1] = 0.0
    f.reshape(-1)[2] = np.inf
    f.reshape(-1)[3] = -np.inf
    f.reshape(-1)[4] = 5e-324                                     # the smallest subnormal
    assert np.array_equal(oracle.order_field_f64(f), _lexsort_rank(f))


def test_order_field_f64_rejects_nan():
    f = np.zeros((4, 5))
    f[2, 3] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.order_field_f64(f)
    assert e.value.code == oracle.ERR_NAN


@pytest.mark.parametrize("mode", ["min", "max", "both"])
def test_f64_equals_f32_on_float32_values(mode):
    rng = np.random.default_rng(11 + len(mode))
    for it in range(40):
        dim3 = it % 2 == 1
        shape = tuple(int(rng.integers(3, 7 if dim3 else 12)) for _ in range(3 if dim3 else 2))
        f32 = rng.integers(0, 7, size=shape).astype(np.float32) * np.float32(0.37)
        O0 = oracle.order_field(f32).reshape(-1)
        ids = np.concatenate([np.nonzero(rng.random(f32.size) < 0.08)[0], [np.argmax(O0), np.argmin(O0)]])
        g32, O32 = oracle.lts(f32, ids, mode)
        g64, O64 = oracle.lts_f64(f32.astype(np.float64), ids, mode)
        assert np.array_equal(O64, O32)
        assert np.array_equal(g64, g32.astype(np.float64))


def test_f64_ties_that_exist_only_in_float32():
    """Values 1 + k * 2^-40 are distinct in float64 and all round to 1.0 in
    float32: the float64 order field is the order of k, the float32 one the
    order of the vertex ids."""
    shape = (6, 8)
    rng = np.random.default_rng(5)
    k = rng.permutation(shape[0] * shape[1]).reshape(shape)
    f = 1.0 + k.astype(np.float64) * 2.0 ** -40
    assert np.all(f.astype(np.float32) == np.float32(1.0))
    assert np.array_equal(oracle.order_field_f64(f), k.astype(np.int32))
    assert np.array_equal(oracle.order_field(f.astype(np.float32)).reshape(-1), np.arange(f.size, dtype=np.int32))
    # the method on it: the extrema of k, the output's extrema exactly the authorized ones
    nbr = H.neighbour_table(shape)
    mins, maxs = H.extrema(k, nbr)
    keep = [min(mins, key=lambda v: k.reshape(-1)[v]), max(maxs, key=lambda v: k.reshape(-1)[v])]
    g, O = oracle.lts_f64(f, np.array(keep, np.int32), "both")
    mins2, maxs2 = H.extrema(O, nbr)
    assert mins2 | maxs2 == set(keep)
    assert np.all(np.isin(g, f))                                  # values are copied, never invented
