"""Writes the stored expected values of the full-size workloads.

Calls only the oracle (and the seeded input generators): for each workload it
records the SHA-256 of the generated field, the authorized extrema selected
by persistence (Sec. 3.3, threshold as a fraction of the range; the global
extrema always kept), and the SHA-256 of the oracle's simplified field g and
order field (mode both: minima pass, then maxima pass) with its statistics.

    python tests/golden/make_golden.py boxnoise3d_512

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


def load_authorized(name):
    """Authorized ids stored by main() (delta-encoded, sorted)."""
    d = np.load(os.path.join(HERE, f"{name}_authorized.npz"))
    return np.cumsum(d["ids"].astype(np.int64)).astype(np.int32)


def load_record(name):
    with open(os.path.join(HERE, f"{name}.json")) as fh:
        return json.load(fh)


if __name__ == "__main__":
    main(sys.argv[1])
