"""Autotuner for the library's launch tuning (lts_set_tuning).

The paper fixes no launch shapes; these are resource choices of this
library.  The tuner times candidate tunings on the GPU and keeps the fastest
per (GPU name, number of dimensions, size bucket) in a JSON cache:

  engine_blocks_per_sm  resident blocks per SM of the persistent propagation
                        engine (its occupancy: more blocks hide more latency,
                        fewer leave room to kernels of other streams);
  team_blocks_per_sm    grid of the 16- and 32-lane local-order team kernels;
  batch_workspaces      workspaces a batch spreads its fields over.

A tuning changes launch shapes only, never a result; the tuner checks that
every candidate reproduces the default tuning's output bit for bit.  A
candidate replaces the current choice only when it is faster by more than
MARGIN (timing noise between candidates is about 1%), so the cache keeps the
defaults where no choice is clearly better.

Per-shape entries are timed on lts_simplify_persistence over a synthetic
field of the bucket's size (every stage of both passes runs, and no
authorized list is needed); batch entries on a caller's batch.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import time

KNOBS = {"engine_blocks_per_sm": (4, 6, 8), "team_blocks_per_sm": (8, 12, 16)}
BATCH_KNOBS = {"batch_workspaces": (8, 16, 32)}
DEFAULTS = {"engine_blocks_per_sm": 8, "team_blocks_per_sm": 12, "batch_workspaces": 32}
MARGIN = 0.02
CACHE_ENV = "LTS_TUNING_CACHE"
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json")


def bucket(shape) -> str:
    """Size bucket of a grid: dimensions and the vertex count rounded up to
    an even power of two (2D and 3D grids of one count differ in
    neighbourhood, so they are tuned apart)."""
    n = int(math.prod(int(d) for d in shape))
    e = max(12, 2 * math.ceil(math.log2(max(n, 2)) / 2))
    return f"{len(shape)}d:2^{e}"


def cache_path(path: str | None = None) -> str:
    return path or os.environ.get(CACHE_ENV) or DEFAULT_CACHE


def load_cache(path: str | None = None) -> dict:
    p = cache_path(path)
    if not os.path.exists(p):
        return {}
    with open(p) as fh:
        return json.load(fh)


def save_cache(cache: dict, path: str | None = None) -> str:
    p = cache_path(path)
    tmp = p + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
        fh.write("\n")
    os.replace(tmp, p)
    return p


def gpu_name(device) -> str:
    import torch

    return torch.cuda.get_device_name(device)


def lookup(cache: dict, gpu: str, key: str) -> dict | None:
    ent = cache.get(gpu, {}).get(key)
    if ent is None:
        return None
    return {k: int(ent[k]) for k in DEFAULTS if k in ent}


def apply(ctx, shape=None, cache: dict | None = None, key: str | None = None, gpu: str | None = None) -> dict:
    """Sets ctx's tuning from the cache entry of the shape's bucket (or of
    `key`, e.g. "batch") for this GPU; the defaults where the cache has none.
    Returns the tuning set."""
    cache = load_cache() if cache is None else cache
    key = key or bucket(shape)
    t = lookup(cache, gpu or gpu_name(ctx.device), key)
    ctx.set_tuning(t)
    return ctx.tuning()


def _time(fn, sync, reps):
    fn()
    sync()
    ts = []
    for _ in range(reps):
        sync()
        t0 = time.perf_counter()
        fn()
        sync()
        ts.append(time.perf_counter() - t0)
    return statistics.median(ts)


def _descend(ctx, knobs, run, same, reps, sync, timer=None, margin=MARGIN):
    """One pass of coordinate descent from the defaults: each knob in turn
    takes the fastest of its candidates (when it beats the current choice by
    more than `margin`), the others held."""
    timer = timer or (lambda fn: _time(fn, sync, reps))
    best = {k: DEFAULTS[k] for k in knobs}
    ctx.set_tuning(best)
    ref = run()
    sync()
    best_t = timer(run)
    trials = [(dict(best), best_t)]
    for k, cands in knobs.items():
        base = dict(best)
        for v in cands:
            if v == base[k]:
                continue
            t = dict(base)
            t[k] = v
            ctx.set_tuning(t)
            out = run()
            sync()
            if not same(ref, out):
                raise RuntimeError(f"tuning {t} changed the result")
            dt = timer(run)
            trials.append((dict(t), dt))
            if dt < best_t * (1.0 - margin):
                best, best_t = t, dt
    ctx.set_tuning(best)
    return best, best_t, trials


def _equal(a, b):
    return all(bool((x == y).all()) for x, y in zip(a, b))


def tune_field(ctx, field, epsilon: float, reps: int = 3, knobs=None):
    """Tunes engine and team grids on one field (lts_simplify_persistence at
    epsilon).  Returns (best tuning, seconds, [(tuning, seconds), ...])."""
    import torch

    knobs = knobs or KNOBS

    def run():
        g, o, _ = ctx.simplify_persistence(field, epsilon, "both", with_stats=False)
        return g.view(torch.int32), o

    return _descend(ctx, knobs, run, _equal, reps, torch.cuda.synchronize)


def tune_batch(ctx, fields, authorized, reps: int = 2, knobs=None):
    """Tunes batch_workspaces on a batch (lists of CUDA tensors)."""
    import torch

    knobs = knobs or BATCH_KNOBS

    def run():
        outs, _ = ctx.simplify_batch(fields, authorized, "both", with_stats=False)
        return [x for g, o in outs for x in (g.view(torch.int32), o)]

    return _descend(ctx, knobs, run, _equal, reps, torch.cuda.synchronize)


def record(cache: dict, gpu: str, key: str, best: dict, seconds: float, trials) -> None:
    ent = dict(DEFAULTS)
    ent.update(best)
    ent["ms"] = round(seconds * 1e3, 3)
    ent["trials"] = [[t, round(s * 1e3, 3)] for t, s in trials]
    cache.setdefault(gpu, {})[key] = ent


def tune_shapes(shapes, device=0, path: str | None = None, reps: int = 3, eps_frac: float = 0.05) -> dict:
    """Tunes the bucket of every shape on the Gaussian-sum recipe (3D shapes
    above 2^24 vertices: the box-noise recipe) and writes the cache."""
    import torch

    import paper_2009_00083_gb300 as lts
    from paper_2009_00083_gb300 import workloads as W

    cache = load_cache(path)
    dev = torch.device("cuda", device)
    gpu = gpu_name(dev)
    for shape in shapes:
        shape = tuple(int(d) for d in shape)
        n = math.prod(shape)
        if len(shape) == 3 and n > (1 << 24):
            f = W.box_noise_field(shape, 2, 1024, W.seed_of(7, n))
        else:
            f = W.gaussian_field(shape, 16 if len(shape) == 2 else 64, 0.05 if len(shape) == 2 else 0.02,
                                 W.seed_of(7, n))
        eps = eps_frac * float(f.max() - f.min())
        fd = torch.from_numpy(f).to(dev)
        ctx = lts.Context(n, device=device)
        try:
            best, sec, trials = tune_field(ctx, fd, eps, reps)
        finally:
            ctx.close()
        record(cache, gpu, bucket(shape), best, sec, trials)
        del fd
        torch.cuda.empty_cache()
    save_cache(cache, path)
    return cache


def main(argv=None):
    import argparse

    ap = argparse.ArgumentParser(description="Tune the library's launch shapes and write the JSON cache.")
    ap.add_argument("--out", default=None, help="cache file (default: $LTS_TUNING_CACHE or the package's)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--shapes", default="256x256,1024x1024,64x64x64,128x128x128,256x256x256,512x512x512",
                    help="comma-separated shapes, one per bucket")
    a = ap.parse_args(argv)
    shapes = [tuple(int(x) for x in s.split("x")) for s in a.shapes.split(",") if s]
    cache = tune_shapes(shapes, path=a.out, reps=a.reps)
    print(json.dumps(cache, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()
