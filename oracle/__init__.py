"""Oracle for Localized Topological Simplification (LTS).

TEST INFRASTRUCTURE ONLY.  A plain single-threaded CPU restatement of the
paper's method (Sections 3-4), written in C (``lts_oracle.c``) and reached
through ctypes.  Only the test-suite, the smoke check and the CPU-baseline
leg of the benchmark may import this package; the CUDA library never does,
and the two share no code.

Public functions (numpy in, numpy out):

    order_field(f)                    Sec. 4.1
    classify(O, shape)                Sec. 3.1 (lower/upper link components)
    persistence(f, O)                 Sec. 3.3 (Elder rule; selector of inputs)
    authorized_by_persistence(f, thr) Sec. 3.3 (the workloads' authorized sets)
    regions(Od, auth, method, seed)   Sec. 4.2 step 1, Sec. 4.3, Sec. 4.4
    local_orders(...)                 Sec. 4.2 step 2 (Eq. 3-5)
    local_order_trace(...)            Sec. 4.2 step 2 on one vertex set, with every intermediate order
    apply(...)                        Sec. 4.2 steps 3-4 (Eq. 6)
    lts(f, auth_ids, mode)            the whole method
    order_field_f64(f), lts_f64(f, auth_ids, mode)   the same on a float64 field
    persistent_by_elder(g, O, dir, eps) Sec. 3.3 as Sec. 4.5 selects (Elder rule, one kind)
    pers_select(f, O, dir, eps)       Sec. 4.5 (propagations from every extremum, stopped at eps)
    pers_lts(f, eps, mode)            Sec. 4.5 (Elder-rule selection per pass, then the pass)
    pers_regions(f, O, dir, eps)      Sec. 4.5 (regions read off the eps-bounded propagations)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lts_oracle.c")
_LIB = os.path.join(_HERE, "liblts_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NAN, ERR_NO_AUTHORIZED, ERR_OOM, ERR_INTERNAL, ERR_CYCLE = 0, 1, 2, 3, 4, 7, 8
MODE_MIN, MODE_MAX, MODE_BOTH = 1, 2, 3
MODE_RESTORE = 4
_MODES = {"min": MODE_MIN, "max": MODE_MAX, "both": MODE_BOTH,
          "min+restore": MODE_MIN | MODE_RESTORE, "max+restore": MODE_MAX | MODE_RESTORE,
          "both+restore": MODE_BOTH | MODE_RESTORE}
# step-2 seeding rules: the adopted one (the paper's alternation, all-boundary
# seeds only for a region where it does not end), the paper's alternation
# alone (ERR_CYCLE where it does not end), all-boundary seeds alone
_RULES = {"adopted": 0, "literal": 1, "boundary": 2}


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [
        ("n_vertices", ctypes.c_int64),
        ("removed", ctypes.c_int64 * 2),
        ("regions", ctypes.c_int64 * 2),
        ("region_vertices", ctypes.c_int64 * 2),
        ("max_region", ctypes.c_int64 * 2),
        ("max_local_floods", ctypes.c_int32 * 2),
        ("pad", ctypes.c_int32),
        ("total_local_floods", ctypes.c_int64 * 2),
        ("fallback_regions", ctypes.c_int64 * 2),
        ("restored", ctypes.c_int64 * 2),
    ]

    def as_dict(self):
        return {
            "n_vertices": self.n_vertices,
            "removed_min": self.removed[0], "removed_max": self.removed[1],
            "regions_min": self.regions[0], "regions_max": self.regions[1],
            "region_vertices_min": self.region_vertices[0],
            "region_vertices_max": self.region_vertices[1],
            "max_region_min": self.max_region[0], "max_region_max": self.max_region[1],
            "max_local_floods_min": self.max_local_floods[0],
            "max_local_floods_max": self.max_local_floods[1],
            "total_local_floods_min": self.total_local_floods[0],
            "total_local_floods_max": self.total_local_floods[1],
            "fallback_regions_min": self.fallback_regions[0],
            "fallback_regions_max": self.fallback_regions[1],
            "restored_min": self.restored[0], "restored_max": self.restored[1],
        }


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, portable flags)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.orc_order_field.argtypes = [ctypes.c_int, P, P, P]
        lib.orc_classify.argtypes = [ctypes.c_int, P, P, P, P]
        lib.orc_persistence.argtypes = [ctypes.c_int, P, P, P, P, P]
        lib.orc_regions.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_uint64, P, P, P, P]
        lib.orc_local_orders.argtypes = [ctypes.c_int, P, P, P, P, i64, P, P]
        lib.orc_local_orders_rule.argtypes = [ctypes.c_int, P, P, P, P, i64, ctypes.c_int, P, P, P]
        lib.orc_local_order_trace.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int,
                                              P, P, P, P, ctypes.c_int32, P]
        lib.orc_order_field_f64.argtypes = [ctypes.c_int, P, P, P]
        lib.orc_lts_f64.argtypes = [ctypes.c_int, P, P, P, i64, ctypes.c_int, P, P, P]
        lib.orc_lts_rule.argtypes = [ctypes.c_int, P, P, P, i64, ctypes.c_int, P, P, P, ctypes.c_int,
                                     ctypes.c_uint64, ctypes.c_int]
        lib.orc_apply.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, P, P]
        lib.orc_lts.argtypes = [ctypes.c_int, P, P, P, i64, ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_uint64]
        lib.orc_pass.argtypes = [ctypes.c_int, P, ctypes.c_int, P, i64, P, P, P, ctypes.c_int, ctypes.c_uint64]
        lib.orc_pers_select.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, P]
        lib.orc_pers_regions.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                         P, P, P, P]
        lib.orc_link_edges.argtypes = [ctypes.c_int, P]
        lib.orc_link_triangles.argtypes = [ctypes.c_int, P]
        lib.orc_neighbour_offsets.argtypes = [ctypes.c_int, P]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(shape):
    """Grid dims (X, Y, Z) from a C-ordered array shape (Z, Y, X) or (Y, X)."""
    if len(shape) == 2:
        return 2, np.array([shape[1], shape[0], 1], dtype=np.int64)
    if len(shape) == 3:
        return 3, np.array([shape[2], shape[1], shape[0]], dtype=np.int64)
    raise ValueError("field must be 2D or 3D")


def _check(code, what):
    if code != OK:
        raise OracleError(code, what)


def neighbour_offsets(ndim):
    off = np.zeros((14, 3), dtype=np.int32)
    k = _get().orc_neighbour_offsets(ndim, _p(off))
    return off[:k, :ndim].copy()


def link_edges(ndim):
    pairs = np.zeros((128, 2), dtype=np.int32)
    e = _get().orc_link_edges(ndim, _p(pairs))
    return pairs[:e].copy()


def link_triangles(ndim):
    tris = np.zeros((512, 3), dtype=np.int32)
    t = _get().orc_link_triangles(ndim, _p(tris))
    return tris[:t].copy()


def order_field(f):
    """Sec. 4.1: rank of every vertex under (value, vertex id)."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    nd, dims = _dims(f.shape)
    O = np.empty(f.shape, dtype=np.int32)
    _check(_get().orc_order_field(nd, _p(dims), _p(f), _p(O)), "order_field")
    return O


def classify(O):
    """Sec. 3.1: (#lower-link components, #upper-link components) per vertex."""
    O = np.ascontiguousarray(O, dtype=np.int32)
    nd, dims = _dims(O.shape)
    lo = np.empty(O.shape, dtype=np.int8)
    up = np.empty(O.shape, dtype=np.int8)
    _check(_get().orc_classify(nd, _p(dims), _p(O), _p(lo), _p(up)), "classify")
    return lo, up


def persistence(f, O=None):
    """Sec. 3.3: persistence of every minimum and maximum (NaN elsewhere)."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    if O is None:
        O = order_field(f)
    nd, dims = _dims(f.shape)
    pmin = np.empty(f.shape, dtype=np.float64)
    pmax = np.empty(f.shape, dtype=np.float64)
    _check(_get().orc_persistence(nd, _p(dims), _p(f), _p(np.ascontiguousarray(O, dtype=np.int32)),
                                  _p(pmin), _p(pmax)), "persistence")
    return pmin, pmax


def authorized_by_persistence(f, thr, O=None):
    """Authorized extrema: persistence strictly above thr * range; the global
    minimum and maximum are always authorized (their persistence is the range)."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    if O is None:
        O = order_field(f)
    pmin, pmax = persistence(f, O)
    rng = float(np.float64(f.max()) - np.float64(f.min()))
    cut = thr * rng
    flat_o = O.reshape(-1)
    keep = np.zeros(f.size, dtype=bool)
    keep |= np.nan_to_num(pmin.reshape(-1), nan=-1.0) > cut
    keep |= np.nan_to_num(pmax.reshape(-1), nan=-1.0) > cut
    keep[int(np.argmin(flat_o))] = True
    keep[int(np.argmax(flat_o))] = True
    return np.nonzero(keep)[0].astype(np.int32)


def regions(Od, auth_mask, method=0, seed=0):
    """Step 1 with hill chains on the pass-oriented order Od (maxima are the
    extrema treated).  Returns (region_of, saddle, top) with regions sorted by
    (Od(saddle), Od(top)); method 0 = propagations, 1 = join-tree sweep."""
    Od = np.ascontiguousarray(Od, dtype=np.int32)
    nd, dims = _dims(Od.shape)
    auth = np.ascontiguousarray(auth_mask.reshape(Od.shape), dtype=np.uint8)
    n = Od.size
    region_of = np.empty(Od.shape, dtype=np.int32)
    sad = np.empty(n, dtype=np.int32)
    top = np.empty(n, dtype=np.int32)
    nreg = np.zeros(1, dtype=np.int64)
    _check(_get().orc_regions(nd, _p(dims), _p(Od), _p(auth), method, seed, _p(region_of), _p(sad), _p(top),
                              _p(nreg)), "regions")
    k = int(nreg[0])
    return region_of, sad[:k].copy(), top[:k].copy()


def local_orders(Od, region_of, saddle, rule="adopted", return_fallback=False):
    """Step 2 for every region: lhat per member vertex (-1 elsewhere), and the
    number of propagations each region needed (with return_fallback, also 1
    for the regions the adopted rule redid with all-boundary seeds)."""
    Od = np.ascontiguousarray(Od, dtype=np.int32)
    nd, dims = _dims(Od.shape)
    lhat = np.empty(Od.shape, dtype=np.int32)
    fl = np.zeros(max(1, len(saddle)), dtype=np.int32)
    fb = np.zeros(max(1, len(saddle)), dtype=np.int32)
    _check(_get().orc_local_orders_rule(nd, _p(dims), _p(Od), _p(np.ascontiguousarray(region_of, dtype=np.int32)),
                                        _p(np.ascontiguousarray(saddle, dtype=np.int32)), len(saddle), _RULES[rule],
                                        _p(lhat), _p(fl), _p(fb)), "local_orders")
    if return_fallback:
        return lhat, fl[:len(saddle)].copy(), fb[:len(saddle)].copy()
    return lhat, fl[:len(saddle)].copy()


def local_order_trace(Od, verts, sidx, rule="adopted", max_trace=64, allow_cycle=False):
    """Step 2 on one vertex set R = verts (the saddle verts[sidx]) of the grid
    of Od.  Returns (lhat over verts, propagations, fell_back, orders) where
    orders[i] is the local order after propagation i of the returned run.
    With allow_cycle, a literal run that does not end returns (None, status,
    False, orders so far) instead of raising."""
    Od = np.ascontiguousarray(Od, dtype=np.int32)
    nd, dims = _dims(Od.shape)
    verts = np.ascontiguousarray(np.asarray(verts, dtype=np.int32).reshape(-1))
    r = verts.size
    lhat = np.empty(r, dtype=np.int32)
    fl = np.zeros(1, dtype=np.int32)
    fb = np.zeros(1, dtype=np.int32)
    tr = np.zeros((max_trace, r), dtype=np.int64)
    nt = np.zeros(1, dtype=np.int32)
    code = _get().orc_local_order_trace(nd, _p(dims), _p(Od), _p(verts), r, int(sidx), _RULES[rule], _p(lhat),
                                        _p(fl), _p(fb), _p(tr), max_trace, _p(nt))
    if allow_cycle and code == ERR_CYCLE:
        return None, code, False, tr[:int(nt[0])].copy()
    _check(code, "local_order_trace")
    return lhat, int(fl[0]), bool(fb[0]), tr[:int(nt[0])].copy()


def apply(Od, region_of, saddle, top, lhat, g):
    """Steps 3-4: the new pass-oriented order and the flattened values."""
    Od = np.ascontiguousarray(Od, dtype=np.int32)
    nd, dims = _dims(Od.shape)
    Od2 = np.empty(Od.shape, dtype=np.int32)
    g2 = np.empty(Od.shape, dtype=np.float32)
    _check(_get().orc_apply(nd, _p(dims), _p(Od), _p(np.ascontiguousarray(region_of, dtype=np.int32)),
                            _p(np.ascontiguousarray(saddle, dtype=np.int32)),
                            _p(np.ascontiguousarray(top, dtype=np.int32)),
                            _p(np.ascontiguousarray(lhat, dtype=np.int32)),
                            _p(np.ascontiguousarray(g, dtype=np.float32)), _p(Od2), _p(g2)), "apply")
    return Od2, g2


def lts(f, auth_ids, mode="both", method=0, seed=0, return_stats=False, rule="adopted"):
    """The whole method: (g, O) after the minima and/or maxima pass.  rule
    picks the step-2 seeding (tests only; the method is "adopted")."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    nd, dims = _dims(f.shape)
    ids = np.ascontiguousarray(np.asarray(auth_ids, dtype=np.int32).reshape(-1))
    g = np.empty(f.shape, dtype=np.float32)
    O = np.empty(f.shape, dtype=np.int32)
    st = Stats()
    code = _get().orc_lts_rule(nd, _p(dims), _p(f), _p(ids) if ids.size else None, ids.size, _MODES[mode],
                               _p(g), _p(O), ctypes.byref(st), method, seed, _RULES[rule])
    _check(code, "lts")
    if return_stats:
        return g, O, st.as_dict()
    return g, O


def order_field_f64(f):
    """Sec. 4.1 on a float64 field: rank of every vertex under (value, vertex id)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    nd, dims = _dims(f.shape)
    O = np.empty(f.shape, dtype=np.int32)
    _check(_get().orc_order_field_f64(nd, _p(dims), _p(f), _p(O)), "order_field_f64")
    return O


def lts_f64(f, auth_ids, mode="both", return_stats=False):
    """The whole method on a float64 field: (g float64, O)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    nd, dims = _dims(f.shape)
    ids = np.ascontiguousarray(np.asarray(auth_ids, dtype=np.int32).reshape(-1))
    g = np.empty(f.shape, dtype=np.float64)
    O = np.empty(f.shape, dtype=np.int32)
    st = Stats()
    code = _get().orc_lts_f64(nd, _p(dims), _p(f), _p(ids) if ids.size else None, ids.size, _MODES[mode],
                              _p(g), _p(O), ctypes.byref(st))
    _check(code, "lts_f64")
    if return_stats:
        return g, O, st.as_dict()
    return g, O


def one_pass(g, O, auth_ids, direction, method=0, seed=0):
    """One pass on a given (g, O): direction +1 maxima, -1 minima."""
    g = np.array(g, dtype=np.float32, copy=True)
    O = np.array(O, dtype=np.int32, copy=True)
    nd, dims = _dims(g.shape)
    ids = np.ascontiguousarray(np.asarray(auth_ids, dtype=np.int32).reshape(-1))
    st = Stats()
    code = _get().orc_pass(nd, _p(dims), direction, _p(ids) if ids.size else None, ids.size, _p(g), _p(O),
                           ctypes.byref(st), method, seed)
    _check(code, "pass")
    return g, O, st.as_dict()


def persistent_by_elder(g, O, direction, eps):
    """Sec. 3.3 applied as Sec. 4.5 selects: the maxima (direction +1) or
    minima (-1) of (g, O) whose Elder-rule persistence exceeds eps, plus the
    global one of that kind."""
    pmin, pmax = persistence(g, O)
    p = (pmax if direction > 0 else pmin).reshape(-1)
    keep = np.nan_to_num(p, nan=-1.0) > eps
    flat = np.asarray(O).reshape(-1)
    keep[int(np.argmax(flat) if direction > 0 else np.argmin(flat))] = True
    return np.nonzero(keep)[0].astype(np.int32)


def pers_select(f, O, direction, eps, seed=0):
    """Sec. 4.5 as the paper runs it: a propagation from every maximum
    (direction +1) or minimum (-1), each ended once its scalar difference to
    the class's highest extremum exceeds eps.  Returns the ids it keeps."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    nd, dims = _dims(f.shape)
    mask = np.empty(f.shape, dtype=np.uint8)
    _check(_get().orc_pers_select(nd, _p(dims), _p(f), _p(np.ascontiguousarray(O, dtype=np.int32)), direction,
                                  float(eps), seed, _p(mask)), "pers_select")
    return np.nonzero(mask.reshape(-1))[0].astype(np.int32)


def pers_lts(f, eps, mode="both"):
    """Persistence-driven LTS (Sec. 4.5): each pass (minima, then maxima)
    keeps the extrema of its kind that are more persistent than eps on the
    field it receives, and simplifies the others."""
    if not (eps >= 0.0):
        raise ValueError("eps must be a non-negative number")
    g = np.array(f, dtype=np.float32, copy=True)
    O = order_field(g)
    if _MODES[mode] & MODE_MIN:
        g, O, _ = one_pass(g, O, persistent_by_elder(g, O, -1, eps), -1)
    if _MODES[mode] & MODE_MAX:
        g, O, _ = one_pass(g, O, persistent_by_elder(g, O, +1, eps), +1)
    return g, O


def pers_regions(f, O, direction, eps, seed=0):
    """The regions of LTS with the persistent extrema authorized, read off
    the eps-bounded propagations of Sec. 4.5 themselves (each merge makes a
    fresh class; the nodes whose extremum is not persistent and that stop at
    a saddle for good, or merge there into a persistent one, are the
    regions).  Returns (region_of, saddle, top) in the order of regions()."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    nd, dims = _dims(f.shape)
    n = f.size
    region_of = np.empty(f.shape, dtype=np.int32)
    sad = np.empty(n, dtype=np.int32)
    top = np.empty(n, dtype=np.int32)
    nreg = np.zeros(1, dtype=np.int64)
    _check(_get().orc_pers_regions(nd, _p(dims), _p(f), _p(np.ascontiguousarray(O, dtype=np.int32)), direction,
                                   float(eps), seed, _p(region_of), _p(sad), _p(top), _p(nreg)), "pers_regions")
    k = int(nreg[0])
    return region_of, sad[:k].copy(), top[:k].copy()
