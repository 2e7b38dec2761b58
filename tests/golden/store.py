"""Readers of the stored expected values under tests/golden (json and numpy
only; the values are written by make_golden.py)."""
from __future__ import annotations

import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load_record(name):
    with open(os.path.join(HERE, f"{name}.json")) as fh:
        return json.load(fh)


def load_authorized(name):
    """Authorized ids of a single-field workload (stored delta-encoded, sorted)."""
    d = np.load(os.path.join(HERE, f"{name}_authorized.npz"))
    return np.cumsum(d["ids"].astype(np.int64)).astype(np.int32)


def load_set_authorized(name):
    """Per-field authorized ids of a multi-field workload."""
    d = np.load(os.path.join(HERE, f"{name}_authorized.npz"))
    off = d["offsets"]
    return [np.cumsum(d["ids"][off[k]:off[k + 1]].astype(np.int64)).astype(np.int32) for k in range(len(off) - 1)]
