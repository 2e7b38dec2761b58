"""Pins of the optional restoration of authorized extrema swallowed by a
flattened region (Sec. 4.2 step 3), as the oracle reads it: after step 2,
each authorized extremum of the other kind inside a region moves below every
other vertex of the region's block (maxima pass; the minima pass mirrors
it), in increasing order, unless one of its neighbours would be left without
a higher neighbour (a new, unauthorized maximum), in which case it stays
swallowed."""
import numpy as np
import pytest

import oracle
from tests import helpers as H


def test_a_swallowed_minimum_is_restored_by_hand():
    """3x3 grid (X = 3, Y = 3), ids x + 3y, authorized 2 (8, the global
    maximum), 4 (0, the global minimum) and 6 (4, a minimum).

        f:  1 2 8      ids: 0 1 2
            5 0 7           3 4 5
            4 6 3           6 7 8

    The maxima pass floods the unauthorized maximum 7 (6): it takes 3 (5) and
    6 (4), then pops 8 (3), whose other higher neighbour 5 (7) is not in the
    class: the region is {7, 3, 6} with saddle 8, and it swallows the
    authorized minimum 6 (its neighbours 7 and 3 are in the region).
    Step 2: inside R the edges are 8-7, 7-3, 7-6, 3-6; 7 is a cut vertex, so
    the minus-infinity vertex is 3; the propagation from 8 visits 8, 7, 6, 3,
    so lhat = (7: 2, 6: 1, 3: 0) and 6 is not a minimum.
    Restoration: 6 moves to the bottom of the block; its neighbours keep a
    higher neighbour (7 has 8, 3 has 7), so it is accepted: lhat = (6: 0,
    3: 1, 7: 2), and 6 is a minimum of the output again."""
    f = np.array([[1, 2, 8], [5, 0, 7], [4, 6, 3]], np.float32)
    ids = np.array([2, 4, 6], np.int32)
    nbr = H.neighbour_table(f.shape)
    g0, O0 = oracle.lts(f, ids, "max")
    g1, O1, st = oracle.lts(f, ids, "max+restore", return_stats=True)
    assert st["restored_max"] == 1
    mins0, maxs0 = H.extrema(O0, nbr)
    mins1, maxs1 = H.extrema(O1, nbr)
    assert mins0 | maxs0 == {2, 4}
    assert mins1 | maxs1 == {2, 4, 6}
    o = O1.reshape(-1)
    assert o[6] < o[3] < o[7] < o[8]                   # the block right below the saddle 8
    assert sorted(o[[6, 3, 7, 8]]) == list(range(o[8] - 3, o[8] + 1))
    assert np.array_equal(g0, g1)                      # only the order changes; values are the saddle's
    assert g1.reshape(-1)[6] == np.float32(3)


def test_a_restoration_that_would_create_a_maximum_is_refused():
    """The 7x4 case of the literal reading: the swallowed authorized minimum 0
    is the only higher neighbour of 1, so moving it down is refused; the
    output keeps only authorized extrema."""
    f = np.array([[15, 22, 8, 13], [16, 21, 0, 24], [14, 3, 10, 11], [2, 27, 1, 18],
                  [12, 5, 25, 9], [23, 20, 6, 4], [19, 17, 7, 26]], np.float32)
    ids = np.array([0, 6, 7, 12, 13, 14, 15, 20, 23], np.int32)
    nbr = H.neighbour_table(f.shape)
    O = oracle.order_field(f)
    g, Og, st = oracle.one_pass(f, O, ids, +1)
    g2, Og2, st2 = oracle.lts(f, ids, "max+restore", return_stats=True)
    assert np.array_equal(Og2, Og) and st2["restored_max"] == 0
    mins, maxs = H.extrema(Og2, nbr)
    assert 0 not in mins and (mins | maxs) <= set(ids.tolist())


@pytest.mark.parametrize("mode", ["min", "max", "both"])
def test_restoration_invariants_on_random_grids(mode):
    rng = np.random.default_rng({"min": 21, "max": 22, "both": 23}[mode])
    restored = 0
    for it in range(150):
        dim3 = it % 3 == 2
        shape = tuple(int(rng.integers(3, 6 if dim3 else 10)) for _ in range(3 if dim3 else 2))
        f = rng.integers(0, 9, size=shape).astype(np.float32) if it % 2 else rng.random(shape).astype(np.float32)
        nbr = H.neighbour_table(shape)
        O = oracle.order_field(f)
        mins, maxs = H.extrema(O, nbr)
        o = O.reshape(-1)
        # arbitrary authorized sets: a random share of the extrema, the global ones always
        ext = sorted(mins | maxs)
        keep = [v for v in ext if rng.random() < 0.5] + [int(np.argmin(o)), int(np.argmax(o))]
        ids = np.array(sorted(set(keep)), np.int32)
        g0, O0 = oracle.lts(f, ids, mode)
        g1, O1, st = oracle.lts(f, ids, mode + "+restore", return_stats=True)
        restored += st["restored_min"] + st["restored_max"]
        assert np.array_equal(g0, g1)                       # the same regions and values
        assert sorted(O1.reshape(-1).tolist()) == list(range(f.size))
        m0, x0 = H.extrema(O0, nbr)
        m1, x1 = H.extrema(O1, nbr)
        A = set(ids.tolist())
        # Eq. 1 for an arbitrary authorized set: the kinds a pass treats keep only authorized extrema
        if mode in ("max", "both"):
            assert x1 <= A
        if mode in ("min", "both"):
            assert m1 <= A
        assert (m0 | x0) <= (m1 | x1)                      # restoring only adds extrema...
        assert ((m1 | x1) - (m0 | x0)) <= A                # ...authorized ones
        assert len((m1 | x1) - (m0 | x0)) == st["restored_min"] + st["restored_max"]
        # every restored vertex changed place
        changed = np.nonzero(O0.reshape(-1) != O1.reshape(-1))[0]
        assert ((m1 | x1) - (m0 | x0)) <= set(changed.tolist())
    assert restored > 0


def test_restoration_changes_nothing_for_persistence_selected_sets():
    from paper_2009_00083_gb300 import workloads as W

    f = W.gaussian_field((64, 48), 8, 0.05, seed=3)
    ids = oracle.authorized_by_persistence(f, 0.05)
    g0, O0 = oracle.lts(f, ids, "both")
    g1, O1, st = oracle.lts(f, ids, "both+restore", return_stats=True)
    assert st["restored_min"] == st["restored_max"] == 0
    assert np.array_equal(O0, O1) and np.array_equal(g0, g1)
