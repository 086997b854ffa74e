"""Seeded synthetic inputs for exact DBSCAN.

This module only draws points; it holds none of the clustering arithmetic, and
both the CUDA path's tests/benchmark and the CPU oracle consume its output.

The paper evaluates on seed-spreader data (SS-simden / SS-varden, 2M points,
d in {2,3,5,7}) and on real sets with every column normalised to integers in
[0, 1e5] (Section 5.1).  The real sets are not available, so these generators
stand in for all workloads:

``blobs``          isotropic Gaussian blobs with centres uniform in the box,
                   plus a fraction of uniform noise.
``seed_spreader``  a random walk that emits ``per_step`` points uniform in a
                   ball of radius ``radius`` around its position, moves
                   ``step`` units in a uniform direction (reflected at the box)
                   and restarts at a uniform position with probability
                   ``restart`` per emitted point; plus uniform noise.
``skewed_mix``     half the points uniform in one eps-ball (the skewed-density
                   worst case), half over Gaussian blobs with sigma
                   log-uniform in a range.

Every generator rounds to the nearest integer, clamps to [0, hi-1] and applies
a seeded random permutation, so the input order carries no spatial locality.
"""
from __future__ import annotations

import numpy as np

HI = 100_000


def _finish(P: np.ndarray, rng: np.random.Generator, hi: int) -> np.ndarray:
    X = np.clip(np.rint(P), 0, hi - 1).astype(np.int32)
    return np.ascontiguousarray(X[rng.permutation(X.shape[0])])


def _in_ball(rng: np.random.Generator, m: int, d: int, radius: float) -> np.ndarray:
    """m points uniform in the d-ball of the given radius, centred at 0."""
    g = rng.standard_normal((m, d))
    g /= np.maximum(np.linalg.norm(g, axis=1, keepdims=True), 1e-300)
    r = radius * rng.random(m) ** (1.0 / d)
    return g * r[:, None]


def blobs(n: int, d: int, k: int = 10, sigma: float = 1500.0, noise: float = 0.05,
          seed: int = 1, hi: int = HI) -> np.ndarray:
    rng = np.random.default_rng(seed)
    n_noise = int(round(n * noise))
    n_blob = n - n_noise
    centres = rng.random((k, d)) * hi
    which = np.arange(n_blob) % k
    P = centres[which] + rng.standard_normal((n_blob, d)) * sigma
    N = rng.random((n_noise, d)) * hi
    return _finish(np.concatenate([P, N]), rng, hi)


def seed_spreader(n: int, d: int, restart: float | None = None, step: float = 50.0,
                  per_step: int = 100, radius: float = 100.0, noise: float = 1e-4,
                  seed: int = 1, hi: int = HI) -> np.ndarray:
    rng = np.random.default_rng(seed)
    if restart is None:
        restart = 10.0 / n
    n_noise = int(round(n * noise))
    n_walk = n - n_noise
    steps = -(-n_walk // per_step)
    pos = np.empty((steps, d))
    x = rng.random(d) * hi
    jump_p = min(1.0, restart * per_step)
    dirs = rng.standard_normal((steps, d))
    dirs /= np.maximum(np.linalg.norm(dirs, axis=1, keepdims=True), 1e-300)
    jumps = rng.random(steps) < jump_p
    targets = rng.random((steps, d)) * hi
    for t in range(steps):
        pos[t] = x
        if jumps[t]:
            x = targets[t].copy()
        else:
            x = x + step * dirs[t]
            x = np.where(x < 0, -x, x)
            x = np.where(x > hi - 1, 2 * (hi - 1) - x, x)
    P = np.repeat(pos, per_step, axis=0)[:n_walk] + _in_ball(rng, n_walk, d, radius)
    N = rng.random((n_noise, d)) * hi
    return _finish(np.concatenate([P, N]), rng, hi)


def skewed_mix(n: int, d: int, eps: float, k: int = 20, sigma_lo: float = 200.0,
               sigma_hi: float = 3000.0, dense_frac: float = 0.5, seed: int = 1,
               hi: int = HI) -> np.ndarray:
    rng = np.random.default_rng(seed)
    n_dense = int(round(n * dense_frac))
    n_blob = n - n_dense
    c0 = eps + rng.random(d) * (hi - 2 * eps)
    D = c0 + _in_ball(rng, n_dense, d, eps)
    centres = rng.random((k, d)) * hi
    sig = np.exp(rng.uniform(np.log(sigma_lo), np.log(sigma_hi), size=k))
    which = np.arange(n_blob) % k
    B = centres[which] + rng.standard_normal((n_blob, d)) * sig[which, None]
    return _finish(np.concatenate([D, B]), rng, hi)


# Named workloads: (generator, eps, MinPts).  eps2 = eps**2 (integers here).
def workload(name: str, seed: int = 1, n: int | None = None):
    """Return (X int32 [n, d], eps2, minpts) for a named workload.

    tiny       d=2, n=20,000: 10 blobs sigma=1500 + 5% noise, eps=800, MinPts=10
    ss3d_2m    d=3, n=2,000,000 seed spreader + 0.01% noise, eps=500, MinPts=20
    ss3d_10m   d=3, n=10,000,000 seed spreader + 0.01% noise, eps=500, MinPts=20
    skew5d_10m d=5, n=10,000,000 skewed mix, eps=1000, MinPts=100
    skew3d_10m d=3, n=10,000,000 skewed mix, eps=500, MinPts=20
    ``n`` overrides the size.  For the seed spreader the restart probability
    stays that of the full workload, so a smaller ``n`` is the same walk
    process stopped early (same local density, fewer points).
    """
    if name == "tiny":
        nn = n or 20_000
        return blobs(nn, 2, k=10, sigma=1500.0, noise=0.05, seed=seed), 800 ** 2, 10
    if name == "ss3d_2m":
        nn = n or 2_000_000
        return seed_spreader(nn, 3, restart=10.0 / 2_000_000, seed=seed), 500 ** 2, 20
    if name == "ss3d_10m":
        nn = n or 10_000_000
        return seed_spreader(nn, 3, restart=10.0 / 10_000_000, seed=seed), 500 ** 2, 20
    if name == "skew5d_10m":
        nn = n or 10_000_000
        return skewed_mix(nn, 5, eps=1000.0, seed=seed), 1000 ** 2, 100
    if name == "skew3d_10m":
        nn = n or 10_000_000
        return skewed_mix(nn, 3, eps=500.0, seed=seed), 500 ** 2, 20
    raise KeyError(name)


def serve_jobs(count: int = 48, seed: int = 1, n_lo: float = 1e3, n_hi: float = 1e7):
    """The serving workload: `count` clustering jobs with n log-uniform in
    [n_lo, n_hi], d uniform in {2, ..., 7}, eps uniform in [200, 2000],
    MinPts uniform in {5, 10, 50, 100}; each job is Gaussian blobs (2 to 8
    blobs, sigma uniform in [300, 3000]) plus 5% uniform noise.
    Returns a list of (X, eps2, minpts)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        d = int(rng.integers(2, 8))
        eps = int(rng.uniform(200, 2000))
        minpts = int(rng.choice([5, 10, 50, 100]))
        X = blobs(n, d, k=int(rng.integers(2, 9)), sigma=float(rng.uniform(300, 3000)), noise=0.05,
                  seed=int(rng.integers(1 << 30)))
        out.append((X, eps * eps, minpts))
    return out


def poisson_arrivals(count: int, rate: float, seed: int = 1) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson stream of `count` requests
    at `rate` per second: cumulative sums of exponential gaps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def batch_instances(k: int = 256, seed: int = 1, n_lo: float = 1e3, n_hi: float = 5e5, only=None):
    """The batched workload: k independent instances with n log-uniform in
    [n_lo, n_hi], d uniform in {2, 3, 5, 7}, eps uniform in [200, 2000],
    MinPts uniform in {5, 10, 50, 100}; each instance is Gaussian blobs (2 to
    8 blobs, sigma uniform in [300, 3000]) plus 5% uniform noise.
    Returns a list of (X, eps2, minpts); with `only` (instance numbers), just
    those instances, identical to their entries in the full list."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        d = int(rng.choice([2, 3, 5, 7]))
        eps = int(rng.uniform(200, 2000))
        minpts = int(rng.choice([5, 10, 50, 100]))
        nblob, sigma, bseed = int(rng.integers(2, 9)), float(rng.uniform(300, 3000)), int(rng.integers(1 << 30))
        if only is not None and i not in only:
            continue
        X = blobs(n, d, k=nblob, sigma=sigma, noise=0.05, seed=bseed)
        out.append((X, eps * eps, minpts))
    return out
