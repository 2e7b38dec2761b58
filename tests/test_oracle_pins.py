"""Pins of the oracle against things other than itself: textbook facts about
the Freudenthal triangulation, a library sort, brute force on tiny grids,
hand-computed examples and the invariants the paper states (Eq. 1, Eq. 3-5,
Sec. 4.2 steps 3-4)."""
import numpy as np
import pytest

import oracle
from paper_2009_00083_gb300 import workloads as W
from tests import helpers as H


# --------------------------------------------------------------------------
# Domain (Sec. 3.1): the link of an interior vertex of the Freudenthal grid
# --------------------------------------------------------------------------

def test_link_2d_is_a_hexagon():
    e = oracle.link_edges(2)
    assert len(oracle.neighbour_offsets(2)) == 6
    assert len(e) == 6
    deg = np.bincount(e.reshape(-1), minlength=6)
    assert np.all(deg == 2)                         # a cycle ...
    seen, stack = {0}, [0]
    while stack:
        v = stack.pop()
        for a, b in e:
            for x, y in ((a, b), (b, a)):
                if x == v and y not in seen:
                    seen.add(y); stack.append(y)
    assert len(seen) == 6                           # ... through all six neighbours


def test_link_3d_is_a_sphere():
    e = oracle.link_edges(3)
    t = oracle.link_triangles(3)
    assert len(oracle.neighbour_offsets(3)) == 14
    assert (len(e), len(t)) == (36, 24)
    assert 14 - len(e) + len(t) == 2                # Euler characteristic of S^2
    # closed surface: every edge lies in exactly two triangles
    edges = {tuple(sorted(x)) for x in e.tolist()}
    cnt = {x: 0 for x in edges}
    for a, b, c in t.tolist():
        for x in ((a, b), (a, c), (b, c)):
            cnt[tuple(sorted(x))] += 1
    assert set(cnt.values()) == {2}
    # the 6 cubes x 6 tetrahedra of the star: 24 link triangles = 24 tetrahedra at a vertex
    off = oracle.neighbour_offsets(3)
    for a, b, c in t.tolist():
        pts = np.array([[0, 0, 0], off[a], off[b], off[c]])
        assert abs(np.linalg.det(pts[1:] - pts[0])) == 1   # unit-volume (1/6) tetrahedra


def test_link_triangulates_unit_cube_into_six():
    """Every tetrahedron with corner 0 in the positive octant is one of the 6
    Kuhn simplices of the unit cube (x_pi1 <= x_pi2 <= x_pi3)."""
    off = oracle.neighbour_offsets(3)
    t = oracle.link_triangles(3)
    pos = [tuple(sorted(tuple(off[i]) for i in tri)) for tri in t.tolist()
           if all(min(off[i]) >= 0 for i in tri)]
    assert len(pos) == 6
    assert all((1, 1, 1) in p for p in pos)


# --------------------------------------------------------------------------
# Order field (Sec. 4.1) against numpy's lexsort
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape,levels", [((7, 9), None), ((5, 6, 7), 4), ((16, 16), 3), ((3, 4, 5), 1)])
def test_order_field_matches_lexsort(shape, levels):
    rng = np.random.default_rng(11)
    f = W.random_tiny_field(rng, shape, levels)
    O = oracle.order_field(f)
    flat = f.reshape(-1).astype(np.float64)
    perm = np.lexsort((np.arange(flat.size), flat))
    ref = np.empty(flat.size, np.int64)
    ref[perm] = np.arange(flat.size)
    assert np.array_equal(O.reshape(-1), ref)


def test_order_field_special_values():
    f = np.array([[0.0, -0.0, 1e-45, -1e-45], [np.inf, -np.inf, 0.0, -0.0]], dtype=np.float32)
    O = oracle.order_field(f).reshape(-1)
    # -inf < -denormal < {0, -0, 0, -0 by id} < denormal < inf
    order = [5, 3, 0, 1, 6, 7, 2, 4]
    assert [int(np.where(O == k)[0][0]) for k in range(8)] == order


def test_order_field_rejects_nan():
    f = np.zeros((4, 4), np.float32)
    f[2, 1] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.order_field(f)
    assert e.value.code == oracle.ERR_NAN


# --------------------------------------------------------------------------
# Critical points (Sec. 3.1, Fig. 2): textbook Morse saddles
# --------------------------------------------------------------------------

def _centre_class(fun, shape):
    if len(shape) == 2:
        y, x = np.mgrid[-1:2, -1:2]
        f = fun(x, y).astype(np.float32)
    else:
        z, y, x = np.mgrid[-1:2, -1:2, -1:2]
        f = fun(x, y, z).astype(np.float32)
    lo, up = oracle.classify(oracle.order_field(f))
    c = tuple(1 for _ in shape)
    return int(lo[c]), int(up[c])


def test_classify_textbook_points():
    assert _centre_class(lambda x, y: x * x + y * y + 0.1 * x, (3, 3)) == (0, 1)        # minimum
    assert _centre_class(lambda x, y: -(x * x + y * y) - 0.1 * x, (3, 3)) == (1, 0)     # maximum
    assert _centre_class(lambda x, y: 1.0 * x + 0.3 * y, (3, 3)) == (1, 1)              # regular
    assert _centre_class(lambda x, y: x * x - y * y + 0.01 * x, (3, 3)) == (2, 2)       # simple saddle
    # 3D: index-1 saddle (lower link S^0, upper link S^1) and index-2 saddle
    assert _centre_class(lambda x, y, z: x * x + y * y - 2.5 * z * z + 0.01 * x, (3, 3, 3)) == (2, 1)
    assert _centre_class(lambda x, y, z: -(x * x + y * y) + 2.5 * z * z + 0.01 * x, (3, 3, 3)) == (1, 2)
    assert _centre_class(lambda x, y, z: x + 0.3 * y + 0.1 * z, (3, 3, 3)) == (1, 1)


def test_monkey_saddle_is_degenerate():
    # Re((x + iy)^3) on the hexagonal link: three lower and three upper sectors
    y, x = np.mgrid[-1:2, -1:2]
    xs = x - 0.5 * y                      # shear the Freudenthal hexagon to a regular one
    ys = y * np.sqrt(3) / 2
    f = (xs ** 3 - 3 * xs * ys * ys + 1e-3 * xs).astype(np.float32)
    lo, up = oracle.classify(oracle.order_field(f))
    assert (int(lo[1, 1]), int(up[1, 1])) == (3, 3)


def test_classify_extrema_match_brute_force():
    rng = np.random.default_rng(3)
    for shape in [(6, 7), (4, 5, 6)]:
        f = W.random_tiny_field(rng, shape)
        O = oracle.order_field(f)
        lo, up = oracle.classify(O)
        nbr = H.neighbour_table(shape)
        mins, maxs = H.extrema(O, nbr)
        assert set(np.nonzero(lo.reshape(-1) == 0)[0]) == mins
        assert set(np.nonzero(up.reshape(-1) == 0)[0]) == maxs


# --------------------------------------------------------------------------
# Persistence (Sec. 3.3) against brute force on tiny grids
# --------------------------------------------------------------------------

def _brute_persistence_max(f, O, nbr):
    o = O.reshape(-1)
    fl = f.reshape(-1).astype(np.float64)
    perm = np.argsort(o)
    _, maxs = H.extrema(O, nbr)
    out = {}
    for m in maxs:
        death = None
        for lam in range(o[m], -1, -1):
            comp = H.component(nbr, m, o >= lam)
            if any(o[w] > o[m] for w in comp):
                death = perm[lam]
                break
        out[m] = None if death is None else fl[m] - fl[death]
    return out


def test_persistence_matches_brute_force():
    rng = np.random.default_rng(5)
    for it in range(12):
        shape = (int(rng.integers(3, 7)), int(rng.integers(3, 7)))
        f = W.random_tiny_field(rng, shape, levels=None if it % 2 else 5)
        O = oracle.order_field(f)
        pmin, pmax = oracle.persistence(f, O)
        nbr = H.neighbour_table(shape)
        ref = _brute_persistence_max(f, O, nbr)
        rng_f = float(f.max()) - float(f.min())
        for m, p in ref.items():
            want = rng_f if p is None else p
            assert pmax.reshape(-1)[m] == pytest.approx(want)
        # minima: the same on -f with the mirrored order
        ref_min = _brute_persistence_max(-f, f.size - 1 - O, nbr)
        for m, p in ref_min.items():
            want = rng_f if p is None else p
            assert pmin.reshape(-1)[m] == pytest.approx(want)


def test_persistence_two_bumps_closed_form():
    # two peaks (3.5 and 2.5) whose only high connection is a col at 1.25 in
    # the middle row; the outer rows stay below 1.  The lower peak dies at the
    # col: persistence 2.5 - 1.25; the global maximum gets the range.
    mid = [0, 1, 3.5, 2, 1.25, 2, 2.5, 1, 0]
    out = [-1, 0, 0.5, 0.5, 0, 0.5, 0.5, 0, -1]
    f = np.array([out, mid, out], np.float32)
    pmin, pmax = oracle.persistence(f)
    assert pmax[1, 2] == pytest.approx(3.5 - (-1.0))
    assert pmax[1, 6] == pytest.approx(2.5 - 1.25)
    assert np.isnan(pmax[1, 4]) and np.isnan(pmax[0, 3])


# --------------------------------------------------------------------------
# Step 1 (Sec. 4.2-4.4): propagations == join-tree sweep == the definition
# --------------------------------------------------------------------------

def _random_case(rng, shape, levels=None, p_auth=0.25):
    f = W.random_tiny_field(rng, shape, levels)
    O = oracle.order_field(f)
    auth = (rng.random(f.size) < p_auth).astype(np.uint8)
    auth[int(np.argmax(O.reshape(-1)))] = 1
    return f, O, auth


@pytest.mark.parametrize("dim3", [False, True])
def test_regions_propagation_equals_jointree_and_definition(dim3):
    rng = np.random.default_rng(21 + dim3)
    for it in range(60):
        shape = tuple(int(rng.integers(2, 6)) for _ in range(3 if dim3 else 2))
        f, O, auth = _random_case(rng, shape, levels=None if it % 3 else 3)
        ra = oracle.regions(O, auth, method=0)
        rb = oracle.regions(O, auth, method=1)
        for a, b in zip(ra, rb):
            assert np.array_equal(a, b)
        region_of, sad, top = ra
        nbr = H.neighbour_table(shape)
        ref = H.brute_regions(O, nbr, auth)
        got = {int(u): int(sad[region_of.reshape(-1)[u]]) for u in np.nonzero(region_of.reshape(-1) >= 0)[0]}
        assert got == ref
        # schedules: shuffled start order and interleaved slices give the same regions
        for seed in (1, 7, 12345):
            rs = oracle.regions(O, auth, method=0, seed=seed)
            for a, b in zip(ra, rs):
                assert np.array_equal(a, b)


def test_regions_hill_chain_merges():
    # two unauthorized peaks joined by a col above the saddle to the authorized peak:
    # one region (hill chain) holding both, stopping at the lower col.
    row = np.array([9, 2, 6, 4, 7, 1, 0], np.float32)
    f = np.stack([row - 0.1, row, row - 0.2]).astype(np.float32)
    O = oracle.order_field(f)
    auth = np.zeros(f.size, np.uint8)
    auth[int(np.argmax(O.reshape(-1)))] = 1
    region_of, sad, top = oracle.regions(O, auth)
    assert len(sad) == 1
    members = set(np.nonzero(region_of.reshape(-1) == 0)[0].tolist())
    cols = {m % 7 for m in members}
    assert cols == {2, 3, 4}                         # both peaks and the col between them
    assert sad[0] % 7 == 1                           # the saddle is on the col at value 2


def test_no_authorized_maximum_is_an_error():
    rng = np.random.default_rng(2)
    f = W.random_tiny_field(rng, (5, 5))
    O = oracle.order_field(f)
    with pytest.raises(oracle.OracleError) as e:
        oracle.regions(O, np.zeros(25, np.uint8))
    assert e.value.code == oracle.ERR_NO_AUTHORIZED


# --------------------------------------------------------------------------
# Step 2 (Eq. 3-5): local orders
# --------------------------------------------------------------------------

def _check_local_orders(O, region_of, sad, lhat, nbr):
    ro = region_of.reshape(-1)
    lh = lhat.reshape(-1)
    o = O.reshape(-1)
    for r, s in enumerate(sad):
        mem = set(np.nonzero(ro == r)[0].tolist())
        R = mem | {int(s)}
        loc = {v: int(lh[v]) for v in mem}
        loc[int(s)] = len(R) - 1
        assert sorted(loc.values()) == list(range(len(R)))
        bnd = {v for v in R if any(u not in R for u in nbr[v])}
        for v in R:
            inside = [u for u in nbr[v] if u in R]
            if all(loc[u] < loc[v] for u in inside):
                assert v == s                       # Eq. 4: s is the only maximum
            if all(loc[u] > loc[v] for u in inside):
                assert v in bnd                     # Eq. 5: minima touch the outside
        assert all(o[v] > o[int(s)] for v in mem)   # a superlevel component above s


@pytest.mark.parametrize("dim3", [False, True])
def test_local_orders_satisfy_eq4_eq5(dim3):
    rng = np.random.default_rng(31 + dim3)
    for it in range(60):
        shape = tuple(int(rng.integers(3, 7 if not dim3 else 5)) for _ in range(3 if dim3 else 2))
        f, O, auth = _random_case(rng, shape, levels=None if it % 2 else 4, p_auth=0.05)
        region_of, sad, top = oracle.regions(O, auth)
        lhat, fl = oracle.local_orders(O, region_of, sad)
        _check_local_orders(O, region_of, sad, lhat, H.neighbour_table(shape))


def test_cut_vertex_is_not_the_minus_infinity_vertex():
    """A 4-vertex region whose lowest boundary vertex is a cut vertex: the
    propagation from s must pass through it, so the minus-infinity vertex is
    the other boundary vertex and the local order is s > 4 > 6 > 7."""
    O = np.array([[6, 7], [2, 1], [3, 0], [4, 5]], np.int32)   # X = 2, Y = 4
    auth = np.zeros(8, np.uint8)
    auth[1] = 1
    region_of, sad, top = oracle.regions(O, auth)
    assert sad.tolist() == [2] and sorted(np.nonzero(region_of.reshape(-1) == 0)[0].tolist()) == [4, 6, 7]
    lhat, fl = oracle.local_orders(O, region_of, sad)
    lh = lhat.reshape(-1)
    assert (lh[4], lh[6], lh[7]) == (2, 1, 0)
    assert fl.tolist() == [1]


def test_single_hill_by_hand():
    """Sec. 4.2 on one hill (I12): 3x5 grid, one unauthorized peak at value 8
    whose saddle is 5; the region is {8, 7, 6} + saddle; the flattened values
    equal the saddle's and the block sits right below it."""
    f = np.array([[0, 1, 2, 3, 4],
                  [1, 9, 5, 7, 6],
                  [2, 3, 4, 8, 1]], np.float32)
    O = oracle.order_field(f)
    auth = np.zeros(f.size, np.uint8)
    auth[int(np.argmax(O.reshape(-1)))] = 1
    auth[int(np.argmin(O.reshape(-1)))] = 1
    g, Og = oracle.lts(f, np.nonzero(auth)[0], mode="max")
    expect = f.copy()
    expect[1, 3] = expect[2, 3] = expect[1, 4] = 5.0
    assert np.array_equal(g, expect)
    o, og = O.reshape(-1), Og.reshape(-1)
    s = 7
    block = sorted([8, 9, 13], key=lambda v: og[v])
    assert [og[v] for v in block] == [og[s] - 3, og[s] - 2, og[s] - 1]
    # vertices outside the region keep their relative order (Eq. 3)
    rest = [v for v in range(15) if v not in (8, 9, 13)]
    assert np.array_equal(np.argsort(o[rest]), np.argsort(og[rest]))


# --------------------------------------------------------------------------
# The whole method: invariants on every output (Eq. 1, Eq. 3, steps 3-4)
# --------------------------------------------------------------------------

def _check_output(f, auth_ids, g, Og, mode, nbr, persistence_selected):
    fo = f.reshape(-1)
    gf = g.reshape(-1)
    og = Og.reshape(-1)
    assert H.is_permutation(og)
    # the order is consistent with the values (step 4)
    srt = np.argsort(og)
    assert np.all(np.diff(gf[srt].astype(np.float64)) >= 0)
    mins, maxs = H.extrema(Og, nbr)
    A = set(int(a) for a in auth_ids)
    if mode in ("max", "both"):
        assert maxs <= A
    if mode in ("min", "both"):
        if mode == "min":
            assert mins <= A
    if persistence_selected and mode == "both":
        assert (mins | maxs) <= A
    if mode == "min":
        assert np.all(gf >= fo)
    if mode == "max":
        assert np.all(gf <= fo)


@pytest.mark.parametrize("mode", ["min", "max", "both"])
def test_lts_invariants_random(mode):
    rng = np.random.default_rng({"min": 41, "max": 42, "both": 43}[mode])
    for it in range(40):
        dim3 = it % 2 == 1
        shape = tuple(int(rng.integers(3, 6 if dim3 else 9)) for _ in range(3 if dim3 else 2))
        f = W.random_tiny_field(rng, shape, levels=None if it % 3 else 6)
        O = oracle.order_field(f)
        ids = np.nonzero(rng.random(f.size) < 0.2)[0]
        ids = np.concatenate([ids, [np.argmax(O.reshape(-1)), np.argmin(O.reshape(-1))]]).astype(np.int32)
        g, Og = oracle.lts(f, ids, mode=mode)
        nbr = H.neighbour_table(shape)
        _check_output(f, ids, g, Og, mode, nbr, False)
        # scheduling does not matter (I11)
        g2, Og2 = oracle.lts(f, ids, mode=mode, seed=99)
        assert np.array_equal(g, g2) and np.array_equal(Og, Og2)
        # propagation (A) and join-tree (B) regions give the same output
        g3, Og3 = oracle.lts(f, ids, mode=mode, method=1)
        assert np.array_equal(g, g3) and np.array_equal(Og, Og3)


def test_lts_persistence_selected_extrema_are_exactly_authorized():
    """Eq. 1 with a persistence selection on the small Gaussian-sum field."""
    f = W.gaussian_field((48, 40), 8, 0.05, seed=7)
    O = oracle.order_field(f)
    ids = oracle.authorized_by_persistence(f, 0.05, O)
    g, Og, st = oracle.lts(f, ids, mode="both", return_stats=True)
    nbr = H.neighbour_table(f.shape)
    mins, maxs = H.extrema(Og, nbr)
    fmins, fmaxs = H.extrema(O, nbr)
    A = set(ids.tolist())
    assert mins | maxs == A & (fmins | fmaxs)
    assert st["removed_min"] > 0 and st["removed_max"] > 0
    _check_output(f, ids, g, Og, "both", nbr, True)
    # error bound of Sec. 4.5: |f - g| <= eps
    rng_f = float(f.max()) - float(f.min())
    assert np.max(np.abs(g.astype(np.float64) - f)) <= 0.05 * rng_f + 1e-7


def test_lts_keeps_everything_when_all_extrema_authorized():
    rng = np.random.default_rng(8)
    f = W.random_tiny_field(rng, (7, 8))
    O = oracle.order_field(f)
    nbr = H.neighbour_table(f.shape)
    mins, maxs = H.extrema(O, nbr)
    g, Og = oracle.lts(f, np.array(sorted(mins | maxs), np.int32), mode="both")
    assert np.array_equal(g, f) and np.array_equal(Og, O)


def test_lts_values_outside_regions_unchanged_and_idempotent():
    f = W.gaussian_field((40, 44), 10, 0.05, seed=3)
    ids = oracle.authorized_by_persistence(f, 0.05)
    g, Og = oracle.lts(f, ids, mode="max")
    O = oracle.order_field(f)
    changed = g != f
    # Eq. 3: relative order of the untouched vertices is preserved
    keep = np.nonzero(~changed.reshape(-1))[0]
    assert np.array_equal(np.argsort(O.reshape(-1)[keep], kind="stable"),
                          np.argsort(Og.reshape(-1)[keep], kind="stable"))
    # the values are a fixed point of the method (I9)
    g2, _ = oracle.lts(g, ids, mode="max")
    assert np.array_equal(g2, g)


def test_lts_rejects_bad_arguments():
    f = np.zeros((4, 4), np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.lts(f, np.array([99], np.int32))
    with pytest.raises(oracle.OracleError):
        oracle.lts(np.zeros((1, 4), np.float32), np.array([0], np.int32))


# --------------------------------------------------------------------------
# Statistics the paper publishes for its experiments (Sec. 5): weak checks
# --------------------------------------------------------------------------

def test_published_statistics_ranges():
    """Step 2 needs one propagation for nearly every region and at most 6;
    a realistic level (1% of the range) processes a small share of a smooth
    3D field; an aggressive level processes up to ~70%."""
    f = W.make_config_field(1)                                   # 128^3 Gaussian sum + noise
    g, O, st = oracle.lts(f, oracle.authorized_by_persistence(f, 0.01), "both", return_stats=True)
    regions = st["regions_min"] + st["regions_max"]
    processed = (st["region_vertices_min"] + st["region_vertices_max"]) / f.size
    assert processed < 0.05
    assert max(st["max_local_floods_min"], st["max_local_floods_max"]) <= 6
    assert (st["total_local_floods_min"] + st["total_local_floods_max"]) / regions < 1.05
    f2 = W.make_config_field(0)                                  # 256^2, noisier
    g2, O2, st2 = oracle.lts(f2, oracle.authorized_by_persistence(f2, 0.05), "both", return_stats=True)
    processed2 = (st2["region_vertices_min"] + st2["region_vertices_max"]) / f2.size
    assert 0.05 < processed2 < 0.75
    assert max(st2["max_local_floods_min"], st2["max_local_floods_max"]) <= 6


def test_region_error_bound_and_flat_value():
    """A maxima pass moves each region's members to the saddle's value, so
    |f - g| <= f(top) - f(saddle) on the region (Sec. 4.2 step 4) and g = f
    elsewhere; the regions come from step 1 on the same input."""
    rng = np.random.default_rng(91)
    for it in range(30):
        dim3 = it % 2 == 1
        shape = tuple(int(rng.integers(3, 7 if dim3 else 14)) for _ in range(3 if dim3 else 2))
        f = W.random_tiny_field(rng, shape, levels=None if it % 3 else 6)
        O = oracle.order_field(f)
        ids = np.nonzero(rng.random(f.size) < 0.15)[0]
        ids = np.concatenate([ids, [np.argmax(O.reshape(-1))]]).astype(np.int32)
        auth = np.zeros(f.size, np.uint8)
        auth[ids] = 1
        region_of, sad, top = oracle.regions(O, auth)
        g, Og, _ = oracle.one_pass(f, O, ids, +1)
        fo, go, ro = f.reshape(-1).astype(np.float64), g.reshape(-1).astype(np.float64), region_of.reshape(-1)
        assert np.array_equal(go[ro < 0], fo[ro < 0])
        for r in range(len(sad)):
            mem = np.nonzero(ro == r)[0]
            assert mem.size > 0
            assert np.all(go[mem] == fo[sad[r]])
            assert np.max(fo[mem] - go[mem]) <= fo[top[r]] - fo[sad[r]]


def test_lowering_a_swallowed_minimum_can_create_a_maximum():
    """Why the optional restoration of swallowed authorized minima (Sec. 4.2)
    needs a reading of its own: on this 7x4 grid the maxima pass swallows the
    authorized minimum a = 0 into a flattened region, and a is the only higher
    neighbour of y = 1 in the output order, so lowering a below its neighbours
    (as the paper suggests) would turn y into a new, unauthorized maximum."""
    f = np.array([[15, 22, 8, 13], [16, 21, 0, 24], [14, 3, 10, 11], [2, 27, 1, 18],
                  [12, 5, 25, 9], [23, 20, 6, 4], [19, 17, 7, 26]], np.float32)
    ids = np.array([0, 6, 7, 12, 13, 14, 15, 20, 23], np.int32)
    nbr = H.neighbour_table(f.shape)
    O = oracle.order_field(f)
    mins, _ = H.extrema(O, nbr)
    assert 0 in mins and 0 in ids
    g, Og, _ = oracle.one_pass(f, O, ids, +1)
    o = Og.reshape(-1)
    mins2, maxs2 = H.extrema(Og, nbr)
    assert 0 not in mins2 and maxs2 <= set(ids.tolist())
    assert [u for u in nbr[1] if o[u] > o[1]] == [0]
