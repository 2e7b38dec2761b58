"""Host-side input generators (no GPU): the output-sensitivity sweep's field
and authorized lists."""
import numpy as np

from paper_2009_00083_gb300 import workloads as W


def test_uniform_noise_field_is_seeded_and_in_range():
    a = W.uniform_noise_field((8, 9, 10), 5)
    b = W.uniform_noise_field((8, 9, 10), 5)
    assert a.dtype == np.float32 and a.shape == (8, 9, 10)
    assert np.array_equal(a, b)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert not np.array_equal(a, W.uniform_noise_field((8, 9, 10), 6))


def test_sweep_authorized_lists():
    f = W.uniform_noise_field((20, 21, 22), 5)
    flat = f.reshape(-1)
    lo, hi = flat.min() - 1.0, flat.max() + 1.0
    flat[[3, 50]] = lo                           # tied minimum: the smaller id is the global one
    flat[[7, 100]] = hi                          # tied maximum: the larger id is the global one
    n = f.size
    gmin, gmax = 3, 100
    shares = (0, 10, 50, 90, 99, 100)
    lists = W.sweep_authorized(f, shares, 77)
    assert len(lists) == len(shares)
    prev = None
    for p, ids in zip(shares, lists):
        assert ids.dtype == np.int32 and np.all(np.diff(ids) > 0)
        assert gmin in ids and gmax in ids
        assert abs((n - ids.size) - min(round(p / 100 * n), n - 2)) <= 2
        if prev is not None:
            assert set(ids.tolist()) <= set(prev.tolist())   # larger shares remove supersets
        prev = ids
    again = W.sweep_authorized(f, shares, 77)
    assert all(np.array_equal(a, b) for a, b in zip(lists, again))
    assert lists[0].size == n
    assert set(lists[-1].tolist()) == {gmin, gmax}
