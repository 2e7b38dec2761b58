"""Seeded synthetic scalar fields standing in for the paper's datasets.

The paper measures on public volumes (Section 5, Table 1) that are not
available here; these generators reproduce their sizes and character:

* ``gaussian_field``: a sum of K Gaussian bumps of random sign plus uniform
  noise (a smooth field with many small noise extrema), 2D or 3D.
* ``uniform_noise_field``: white noise, independent U[0, 1) samples (the
  random dataset of the output-sensitivity sweep, Fig. 6).
* ``box_noise_field``: white noise box-filtered with radius r and quantized to
  1024 levels, so that many neighbouring vertices tie and the order field has
  to break ties by vertex id (Section 4.1).

Every array is C-ordered with shape (Z, Y, X) (3D) or (Y, X) (2D), so the
flat index is the vertex id ``x + X*(y + Y*z)``.  Randomness comes from
``numpy.random.Generator(PCG64(seed))`` only, in a fixed draw order, so a
field is identical on every platform.  This module holds input generation
only: nothing here computes an order field, an extremum or a region.
"""
from __future__ import annotations

import hashlib
import math

import numpy as np

#: (name, shape, persistence threshold as a fraction of the range)
CONFIGS = {
    0: dict(name="gauss2d_256", shape=(256, 256), K=16, noise=0.05, thr=0.05, kind="gauss"),
    1: dict(name="gauss3d_128", shape=(128, 128, 128), K=64, noise=0.02, thr=0.01, kind="gauss"),
    2: dict(name="boxnoise3d_512", shape=(512, 512, 512), radius=2, levels=1024, thr=0.10, kind="box"),
    # many fields at once: even k a 2D square of side exp(U[ln 64, ln 1024]), odd k a 3D cube of side
    # exp(U[ln 32, ln 160]); the Gaussian-sum generator of gauss2d_256; threshold U[1%, 10%] per field
    3: dict(name="mixed_batch_256", count=256, K=16, noise=0.05, kind="batch"),
    # served requests: 3D cubes of side exp(U[ln 32, ln 256]); the Gaussian-sum generator of gauss3d_128; threshold
    # U[0.5%, 10%] per request; Poisson arrivals at 200/s
    4: dict(name="serve_3d", K=64, noise=0.02, rate_hz=200.0, kind="serve"),
}


def seed_of(config: int, k: int = 0) -> int:
    return 1000 * config + k


def _coords(n):
    return np.arange(n, dtype=np.float64) / float(n - 1)


def gaussian_field(shape, K, noise, seed, sigma=(0.05, 0.15), amp=(0.5, 1.0), dtype=np.float32):
    """sum_k a_k exp(-|p - c_k|^2 / (2 sigma_k^2)) + U[-noise, noise], computed in
    float64 and returned as `dtype` (float32 unless asked for float64).

    Draw order: centres (K x d), sigma (K), |a| (K), signs (K), noise (N, x fastest).
    Coordinates are idx / (dim - 1), so the extent is the unit square or cube."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = len(shape)
    centres = rng.random((K, d))
    sig = rng.uniform(sigma[0], sigma[1], K)
    mag = rng.uniform(amp[0], amp[1], K)
    sign = np.where(rng.random(K) < 0.5, -1.0, 1.0)
    n = int(np.prod(shape))
    eps = rng.uniform(-noise, noise, n) if noise > 0 else np.zeros(n)
    # axes in (x, y[, z]) order against shape (.., Y, X)
    axes = [_coords(s) for s in reversed(shape)]
    f = np.zeros(shape, dtype=np.float64)
    for k in range(K):
        # separable: exp(-sum_i (p_i - c_i)^2 / 2s^2) = prod_i exp(-(p_i - c_i)^2 / 2s^2)
        parts = [np.exp(-((axes[i] - centres[k, i]) ** 2) / (2.0 * sig[k] ** 2)) for i in range(d)]
        if d == 2:
            term = parts[1][:, None] * parts[0][None, :]
        else:
            term = parts[2][:, None, None] * parts[1][None, :, None] * parts[0][None, None, :]
        f += sign[k] * mag[k] * term
    f += eps.reshape(shape)
    return f.astype(dtype)


def _box_sum_axis(a, axis, r):
    """Sum over the in-bounds window [i-r, i+r] along one axis, and its width."""
    n = a.shape[axis]
    c = np.cumsum(a, axis=axis, dtype=np.int64)
    pad_shape = list(a.shape)
    pad_shape[axis] = 1
    c = np.concatenate([np.zeros(pad_shape, dtype=np.int64), c], axis=axis)
    i = np.arange(n)
    hi = np.minimum(i + r + 1, n)
    lo = np.maximum(i - r, 0)
    s = np.take(c, hi, axis=axis) - np.take(c, lo, axis=axis)
    return s, (hi - lo)


def box_noise_field(shape, radius, levels, seed, bits=24):
    """White noise U[0,1) (drawn as `bits`-bit fixed point, so box sums are
    exact integers), box mean over the in-bounds part of the (2r+1)^d box,
    quantized as q = min(levels-1, floor(levels*(v-min)/(max-min))) and stored
    as q/(levels-1) in float32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(np.prod(shape))
    w = rng.integers(0, 1 << bits, size=n, dtype=np.int64).reshape(shape)
    cnt = np.ones(shape, dtype=np.int64)
    s = w
    for ax in range(len(shape)):
        s, width = _box_sum_axis(s, ax, radius)
        bshape = [1] * len(shape)
        bshape[ax] = shape[ax]
        cnt = cnt * width.reshape(bshape)
    del w
    v = s.astype(np.float64) / (cnt.astype(np.float64) * float(1 << bits))
    del s, cnt
    vmin, vmax = float(v.min()), float(v.max())
    if vmax > vmin:
        q = np.floor(levels * (v - vmin) / (vmax - vmin))
    else:
        q = np.zeros_like(v)
    np.minimum(q, levels - 1, out=q)
    return (q / float(levels - 1)).astype(np.float32)


def uniform_noise_field(shape, seed):
    """White noise: independent U[0, 1) samples as float32 (the random field of
    the output-sensitivity sweep)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random(int(np.prod(shape)), dtype=np.float32).reshape(shape)


def sweep_authorized(f, removed_pcts, seed):
    """Authorized lists of the output-sensitivity sweep, one per share in
    removed_pcts: every vertex except a random share of them (a prefix of one
    seeded permutation, so larger shares remove supersets), never the global
    minimum or maximum under (value, id) order; ids ascending, int32."""
    flat = np.asarray(f).reshape(-1)
    n = flat.size
    keep = np.array([int(np.flatnonzero(flat == flat.min()).min()), int(np.flatnonzero(flat == flat.max()).max())])
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = rng.permutation(n)
    perm = perm[(perm != keep[0]) & (perm != keep[1])]
    out = []
    for p in removed_pcts:
        drop = min(int(round(p / 100.0 * n)), perm.size)
        mask = np.ones(n, dtype=bool)
        mask[perm[:drop]] = False
        mask[keep] = True
        out.append(np.flatnonzero(mask).astype(np.int32))
    return out


def make_config_field(config: int, k: int = 0, shape=None):
    """The field of a numbered configuration (optionally at another shape)."""
    c = CONFIGS[config]
    shp = tuple(shape) if shape is not None else c["shape"]
    s = seed_of(config, k)
    if c["kind"] == "gauss":
        return gaussian_field(shp, c["K"], c["noise"], s)
    return box_noise_field(shp, c["radius"], c["levels"], s)


def random_tiny_field(rng: np.random.Generator, shape, levels=None):
    """Small test fields: a random permutation (no ties) or `levels` distinct
    values (heavy ties), float32."""
    n = int(np.prod(shape))
    if levels is None:
        return rng.permutation(n).astype(np.float32).reshape(shape)
    return rng.integers(0, levels, size=n).astype(np.float32).reshape(shape)


def sha256_of(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def dims_of(shape):
    """(ndim, (X, Y, Z)) of a C-ordered field shape."""
    if len(shape) == 2:
        return 2, (shape[1], shape[0], 1)
    return 3, (shape[2], shape[1], shape[0])


def log_uniform_int(rng, lo, hi):
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def batch_specs(count=256):
    """Shapes, thresholds and seeds of the fields of the batch workload
    (mixed_batch_256), drawn in field order from their own generator."""
    rng = np.random.Generator(np.random.PCG64(seed_of(3, 999)))
    specs = []
    for k in range(count):
        if k % 2 == 0:
            side = int(round(float(np.exp(rng.uniform(np.log(64.0), np.log(1024.0))))))
            shape = (side, side)
        else:
            side = int(round(float(np.exp(rng.uniform(np.log(32.0), np.log(160.0))))))
            shape = (side, side, side)
        specs.append(dict(shape=shape, thr=float(rng.uniform(0.01, 0.10)), seed=seed_of(3, k)))
    return specs


def batch_field(spec):
    c = CONFIGS[3]
    return gaussian_field(spec["shape"], c["K"], c["noise"], spec["seed"])


def serve_specs(count):
    """Shapes, thresholds and seeds of served requests (serve_3d)."""
    rng = np.random.Generator(np.random.PCG64(seed_of(4, 999)))
    specs = []
    for k in range(count):
        side = int(round(float(np.exp(rng.uniform(np.log(32.0), np.log(256.0))))))
        specs.append(dict(shape=(side, side, side), thr=float(rng.uniform(0.005, 0.10)), seed=seed_of(4, k)))
    return specs


def serve_field(spec):
    c = CONFIGS[4]
    return gaussian_field(spec["shape"], c["K"], c["noise"], spec["seed"])


def serve_arrivals(count, rate_hz=200.0):
    """Arrival times (seconds from the first) of a Poisson process."""
    rng = np.random.Generator(np.random.PCG64(seed_of(4, 998)))
    gaps = rng.exponential(1.0 / rate_hz, count)
    gaps[0] = 0.0
    return np.cumsum(gaps)
