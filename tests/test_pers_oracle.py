"""Pins of the persistence-driven oracle (Sec. 4.5).

* The propagations started from every extremum and ended once the scalar
  difference to their class's highest extremum exceeds eps (the paper's
  procedure, ``oracle.pers_select``) keep exactly the extrema whose Elder-rule
  persistence exceeds eps, plus the global one (``persistent_by_elder``, whose
  persistence is pinned against brute force elsewhere), under any schedule.
* A two-peak field worked by hand, on both sides of the threshold.
* The guarantee the paper states: |f - g| <= eps everywhere, and the extrema
  left by each pass are exactly the ones it selected.
"""
import numpy as np
import pytest

import oracle
from paper_2009_00083_gb300 import workloads as W
from tests import helpers as H


def _eps_choices(f, O, rng):
    pmin, pmax = oracle.persistence(f, O)
    p = np.concatenate([pmin[~np.isnan(pmin)], pmax[~np.isnan(pmax)]])
    rngf = float(np.float64(f.max()) - np.float64(f.min()))
    # exact persistence values (p == eps must not be kept), values between them, 0, beyond the range
    return [0.0, float(rng.choice(p)), float(rng.choice(p)), float(np.median(p)), 0.37 * rngf, 2.0 * rngf + 1.0]


@pytest.mark.parametrize("dim3", [False, True])
def test_propagations_select_exactly_the_elder_rule_set(dim3):
    rng = np.random.default_rng(451 + dim3)
    for it in range(50):
        shape = tuple(int(rng.integers(2, 7 if dim3 else 12)) for _ in range(3 if dim3 else 2))
        f = W.random_tiny_field(rng, shape, levels=None if it % 3 else 4)
        O = oracle.order_field(f)
        for eps in _eps_choices(f, O, rng):
            for d in (1, -1):
                want = oracle.persistent_by_elder(f, O, d, eps)
                for seed in (0, 7, 1234):
                    got = oracle.pers_select(f, O, d, eps, seed=seed)
                    assert np.array_equal(got, want), (it, shape, eps, d, seed)


def test_propagations_select_on_a_smooth_field_with_infinities():
    f = W.gaussian_field((40, 36), 8, 0.05, seed=3)
    f[5, 7] = np.inf
    f[5, 8] = np.inf
    f[30, 30] = -np.inf
    O = oracle.order_field(f)
    for eps in (0.0, 0.01, 0.05, 0.2, float("inf")):
        for d in (1, -1):
            assert np.array_equal(oracle.pers_select(f, O, d, eps, seed=5), oracle.persistent_by_elder(f, O, d, eps))


# two peaks (3.5 and 2.5) joined by a col at 1.25 in the middle row; the
# outer rows stay below 1.  The lower peak's hill above the col is
# {(1,5), (1,6)}: its persistence is 2.5 - 1.25 = 1.25 exactly.
MID = [0, 1, 3.5, 2, 1.25, 2, 2.5, 1, 0]
OUT = [-1, 0, 0.5, 0.5, 0, 0.5, 0.5, 0, -1]


def test_two_peaks_by_hand():
    f = np.array([OUT, MID, OUT], np.float32)
    # at eps = 1.25 the lower peak is not more persistent than eps: flattened to the col
    g, O = oracle.pers_lts(f, 1.25, mode="max")
    want = f.copy()
    want[1, 5] = want[1, 6] = 1.25
    assert np.array_equal(g, want)
    # just below, it stays; far above, the same hill goes
    g, O = oracle.pers_lts(f, np.nextafter(1.25, 0.0), mode="max")
    assert np.array_equal(g, f)
    g, O = oracle.pers_lts(f, 4.0, mode="max")
    assert np.array_equal(g, want)
    # the global maximum is always kept, even with eps beyond the range
    g, O = oracle.pers_lts(f, 100.0, mode="max")
    assert g[1, 2] == np.float32(3.5) and np.array_equal(g, want)


@pytest.mark.parametrize("mode", ["min", "max", "both"])
def test_error_bound_and_remaining_extrema(mode):
    rng = np.random.default_rng({"min": 61, "max": 62, "both": 63}[mode])
    for it in range(24):
        dim3 = it % 2 == 1
        shape = tuple(int(rng.integers(3, 7 if dim3 else 14)) for _ in range(3 if dim3 else 2))
        f = W.random_tiny_field(rng, shape, levels=None if it % 3 else 5) if it % 4 else \
            W.gaussian_field(shape, 4, 0.1, seed=int(rng.integers(1 << 30)))
        rngf = float(np.float64(f.max()) - np.float64(f.min()))
        eps = float(rng.uniform(0.0, 0.5)) * rngf
        g, Og = oracle.pers_lts(f, eps, mode=mode)
        # Sec. 4.5: ||f - g||_inf <= eps
        assert np.max(np.abs(g.astype(np.float64) - f.astype(np.float64))) <= eps
        # every pass leaves exactly the extrema it selected (Eq. 1)
        nbr = H.neighbour_table(shape)
        gm = f.copy()
        Om = oracle.order_field(f)
        if mode in ("min", "both"):
            sel = oracle.persistent_by_elder(gm, Om, -1, eps)
            gm, Om, _ = oracle.one_pass(gm, Om, sel, -1)
            assert H.extrema(Om, nbr)[0] == set(sel.tolist())
        if mode in ("max", "both"):
            sel = oracle.persistent_by_elder(gm, Om, +1, eps)
            gm, Om, _ = oracle.one_pass(gm, Om, sel, +1)
            assert H.extrema(Om, nbr)[1] == set(sel.tolist())
        assert np.array_equal(gm, g) and np.array_equal(Om, Og)


def test_large_eps_leaves_one_minimum_and_one_maximum():
    f = W.gaussian_field((30, 26), 8, 0.05, seed=11)
    g, Og = oracle.pers_lts(f, 10.0, mode="both")
    mins, maxs = H.extrema(Og, H.neighbour_table(f.shape))
    assert len(mins) == 1 and len(maxs) == 1


def test_zero_eps_keeps_every_extremum_of_a_field_without_ties():
    rng = np.random.default_rng(5)
    f = W.random_tiny_field(rng, (9, 10))
    g, Og = oracle.pers_lts(f, 0.0, mode="both")
    assert np.array_equal(g, f) and np.array_equal(Og, oracle.order_field(f))


def test_negative_or_nan_eps_is_rejected():
    f = np.zeros((3, 3), np.float32)
    with pytest.raises(ValueError):
        oracle.pers_lts(f, -1.0)
    with pytest.raises(ValueError):
        oracle.pers_lts(f, float("nan"))


@pytest.mark.parametrize("dim3", [False, True])
def test_regions_read_off_the_selection_equal_lts_regions(dim3):
    """A single-phase formulation of Sec. 4.5: the regions of LTS with the
    persistent extrema authorized can be read off the eps-bounded
    propagations (with a fresh class per merge), under any schedule."""
    rng = np.random.default_rng(811 + dim3)
    for it in range(40):
        shape = tuple(int(rng.integers(2, 7 if dim3 else 12)) for _ in range(3 if dim3 else 2))
        f = W.random_tiny_field(rng, shape, levels=None if it % 3 else 4)
        O = oracle.order_field(f)
        n = f.size
        for eps in _eps_choices(f, O, rng):
            for d in (1, -1):
                keep = oracle.pers_select(f, O, d, eps)
                auth = np.zeros(n, np.uint8)
                auth[keep] = 1
                Od = O if d > 0 else (n - 1 - O)
                want = oracle.regions(Od, auth)
                for seed in (0, 5):
                    got = oracle.pers_regions(f, O, d, eps, seed=seed)
                    assert np.array_equal(got[0], want[0]), (it, shape, eps, d, seed)
                    assert np.array_equal(got[1], want[1]) and np.array_equal(got[2], want[2])
