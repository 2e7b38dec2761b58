"""Writes the stored expected values of the full-size workloads.

Calls only the oracle (and the seeded input generators): for each workload it
records the SHA-256 of the generated field, the authorized extrema selected
by persistence (Sec. 3.3, threshold as a fraction of the range; the global
extrema always kept), and the SHA-256 of the oracle's simplified field g and
order field (mode both: minima pass, then maxima pass) with its statistics.

    python tests/golden/make_golden.py boxnoise3d_512
    python tests/golden/make_golden.py mixed_batch_256    # the mixed batch, 256 fields
    python tests/golden/make_golden.py serve_pool_16      # served requests, the first 16
    python tests/golden/make_golden.py pers boxnoise3d_512   # persistence-driven (Sec. 4.5)
    python tests/golden/make_golden.py sweep 256          # the output-sensitivity sweep (Fig. 6)

The persistence-driven records ({name}_pers.json) hold, for eps = thr * range
of the field (range = max - min in double precision), the hashes of the
oracle's pers_lts output (mode both) and the number of extrema each pass keeps.

The GPU tests regenerate the field, check its hash, run the library with the
stored authorized list and compare the hashes of its outputs; bench.py uses
the stored authorized list.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2009_00083_gb300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
TARGETS = {
    "boxnoise3d_512": (2, None),
    "boxnoise3d_256": (2, (256, 256, 256)),
}


def main(name):
    cfg, shape = TARGETS[name]
    t0 = time.time()
    f = W.make_config_field(cfg, shape=shape)
    fsha = W.sha256_of(f)
    t1 = time.time()
    O = oracle.order_field(f)
    ids = oracle.authorized_by_persistence(f, W.CONFIGS[cfg]["thr"], O)
    t2 = time.time()
    g, Og, st = oracle.lts(f, ids, mode="both", return_stats=True)
    t3 = time.time()
    np.savez_compressed(os.path.join(HERE, f"{name}_authorized.npz"),
                        ids=np.diff(np.concatenate([[0], np.sort(ids)])).astype(np.int32))
    rec = {
        "workload": name, "config": cfg, "shape": list(f.shape), "thr": W.CONFIGS[cfg]["thr"],
        "field_sha256": fsha, "n_authorized": int(ids.size),
        "g_sha256": W.sha256_of(g), "order_sha256": W.sha256_of(Og),
        "stats": st,
        "oracle_seconds": {"generate": round(t1 - t0, 1), "order_and_persistence": round(t2 - t1, 1),
                           "lts_both": round(t3 - t2, 1)},
    }
    with open(os.path.join(HERE, f"{name}.json"), "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps(rec, indent=1))


SETS = {"mixed_batch_256": ("batch", 256), "serve_pool_16": ("serve", 16)}


def _specs(name):
    kind, count = SETS[name]
    return W.batch_specs(count) if kind == "batch" else W.serve_specs(count)


def _one_field(args):
    name, k = args
    kind, _ = SETS[name]
    spec = _specs(name)[k]
    f = W.batch_field(spec) if kind == "batch" else W.serve_field(spec)
    O = oracle.order_field(f)
    ids = oracle.authorized_by_persistence(f, spec["thr"], O)
    g, Og = oracle.lts(f, ids, mode="both")
    return k, W.sha256_of(f), np.sort(ids).astype(np.int64), W.sha256_of(g), W.sha256_of(Og)


def main_set(name, procs=8):
    """A set of fields (one record each): field hash, authorized ids, output hashes."""
    import multiprocessing as mp

    specs = _specs(name)
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        res = sorted(pool.map(_one_field, [(name, k) for k in range(len(specs))], chunksize=1))
    ids = [r[2] for r in res]
    off = np.cumsum([0] + [len(i) for i in ids])
    flat = np.concatenate([np.diff(np.concatenate([[0], i])) for i in ids]).astype(np.int32)
    np.savez_compressed(os.path.join(HERE, f"{name}_authorized.npz"), ids=flat, offsets=off.astype(np.int64))
    rec = {"workload": name, "fields": [
        {"shape": list(spec["shape"]), "thr": spec["thr"], "seed": spec["seed"], "field_sha256": r[1],
         "n_authorized": int(len(r[2])), "g_sha256": r[3], "order_sha256": r[4]}
        for spec, r in zip(specs, res)], "oracle_seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, f"{name}.json"), "w") as fh:
        json.dump(rec, fh, indent=0)
    print(name, len(specs), "fields,", int(off[-1]), "authorized ids,", rec["oracle_seconds"], "s")


def main_pers(name):
    """Persistence-driven LTS (Sec. 4.5) on a single-field workload."""
    cfg, shape = TARGETS[name]
    t0 = time.time()
    f = W.make_config_field(cfg, shape=shape)
    thr = W.CONFIGS[cfg]["thr"]
    eps = thr * float(np.float64(f.max()) - np.float64(f.min()))
    g = f.copy()
    O = oracle.order_field(f)
    kept = []
    for d in (-1, 1):
        ids = oracle.persistent_by_elder(g, O, d, eps)
        kept.append(int(ids.size))
        g, O, _ = oracle.one_pass(g, O, ids, d)
    rec = {"workload": name, "config": cfg, "shape": list(f.shape), "thr": thr, "eps": eps,
           "field_sha256": W.sha256_of(f), "kept_min": kept[0], "kept_max": kept[1],
           "g_sha256": W.sha256_of(g), "order_sha256": W.sha256_of(O),
           "max_abs_change": float(np.max(np.abs(g.astype(np.float64) - f))),
           "oracle_seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, f"{name}_pers.json"), "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps(rec, indent=1))


SWEEP_POINTS = (0, 50, 90, 99, 100)


def main_sweep(side=256):
    """The output-sensitivity sweep (Fig. 6): uniform white noise on side^3,
    a random share p of the vertices left out of an otherwise complete
    authorized list (workloads.sweep_authorized); the oracle's output hashes
    and statistics per share (mode both)."""
    t0 = time.time()
    f = W.uniform_noise_field((side,) * 3, W.seed_of(5))
    lists = W.sweep_authorized(f, SWEEP_POINTS, W.seed_of(5, 1))
    pts = []
    for p, ids in zip(SWEEP_POINTS, lists):
        g, O, st = oracle.lts(f, ids, mode="both", return_stats=True)
        pts.append({"removed_pct": p, "n_authorized": int(ids.size), "g_sha256": W.sha256_of(g),
                    "order_sha256": W.sha256_of(O), "stats": st})
    rec = {"workload": f"sweep_{side}", "shape": [side] * 3, "field_sha256": W.sha256_of(f), "points": pts,
           "oracle_seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, f"sweep_{side}.json"), "w") as fh:
        json.dump(rec, fh, indent=1)
    print(f"sweep_{side}", rec["oracle_seconds"], "s")


from tests.golden.store import load_authorized, load_record, load_set_authorized  # noqa: E402,F401


if __name__ == "__main__":
    if sys.argv[1] == "pers":
        main_pers(sys.argv[2])
    elif sys.argv[1] == "sweep":
        main_sweep(int(sys.argv[2]) if len(sys.argv) > 2 else 256)
    elif sys.argv[1] in SETS:
        main_set(sys.argv[1])
    else:
        main(sys.argv[1])
