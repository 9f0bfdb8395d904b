"""Seeded synthetic workloads for the KAFMM evaluation.

This module only draws random inputs; it holds none of the method's arithmetic, so both the
CPU oracle and the CUDA path can consume the same arrays.  Every workload lives in the unit
cube [0,1)^3 (the paper uses [0,L)^3 with L = 32, Sec. III; the kernels are homogeneous, so
scaling the box is exact).

Recipes (numpy PCG64 ``default_rng``; points are drawn first, then values):

* ``laplace_uniform``  -- N uniform points, FP64, charges s ~ U(-1, 1).
* ``stokes_uniform``   -- N uniform points, forces f ~ N(0, 1)^3, optional FP32 cast and
  optional mean removal (zero net force, needed by the triply periodic sum).
* ``rpy_clusters``     -- N points in ``n_clusters`` Gaussian clusters (centres uniform in the
  cube, standard deviation ``sigma``), clipped into the cube, radii a ~ U(a_lo, a_hi),
  forces f ~ N(0, 1)^3.
* ``batched_sizes``    -- problem sizes N_k = floor(exp(U(ln lo, ln hi))); problem k draws
  from ``default_rng([seed, k])``.
* ``lognormal_points`` -- the paper's own benchmark cloud (Eq. ptdist, Sec. III): each
  coordinate is the fractional part of a log-normal variate (m = -1, s = 0.5).
"""
from __future__ import annotations

import numpy as np

# largest FP32 / FP64 values strictly below 1.0, used to clip points into [0, 1)
_BELOW_ONE = {np.float32: np.float32(1.0) - np.float32(2.0 ** -24),
              np.float64: 1.0 - 2.0 ** -53}


def _cast(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a.astype(dtype, copy=False))


def _clip_unit(p: np.ndarray) -> np.ndarray:
    hi = _BELOW_ONE[p.dtype.type]
    return np.clip(p, p.dtype.type(0), hi)


def laplace_uniform(n: int, seed: int = 0, dtype=np.float64):
    """Uniform points in [0,1)^3 and scalar charges U(-1, 1)."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    s = rng.uniform(-1.0, 1.0, (n, 1))
    return _clip_unit(_cast(pts, dtype)), _cast(s, dtype)


def stokes_uniform(n: int, seed: int = 1, dtype=np.float32, zero_mean: bool = False):
    """Uniform points in [0,1)^3 and Gaussian forces N(0,1)^3 (optionally mean-free)."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    f = rng.standard_normal((n, 3))
    if zero_mean:
        f = f - f.mean(axis=0, keepdims=True)
    return _clip_unit(_cast(pts, dtype)), _cast(f, dtype)


def rpy_clusters(n: int, seed: int = 2, n_clusters: int = 64, sigma: float = 0.02,
                 a_lo: float = 0.002, a_hi: float = 0.006, dtype=np.float32):
    """Gaussian-clustered points, per-point radii and Gaussian forces.

    Returns (points [n,3], forces [n,3], radii [n]).  Points are assigned to clusters
    round-robin in blocks of n // n_clusters (the remainder goes to the last cluster).
    """
    rng = np.random.default_rng(seed)
    centres = rng.random((n_clusters, 3))
    per = n // n_clusters
    owner = np.minimum(np.arange(n) // max(per, 1), n_clusters - 1)
    pts = centres[owner] + sigma * rng.standard_normal((n, 3))
    pts = np.clip(pts, 0.0, _BELOW_ONE[np.float64])
    a = rng.uniform(a_lo, a_hi, n)
    f = rng.standard_normal((n, 3))
    return _clip_unit(_cast(pts, dtype)), _cast(f, dtype), _cast(a, dtype)


def batched_sizes(n_prob: int = 512, lo: int = 1024, hi: int = 65536, seed: int = 3):
    """Log-uniform problem sizes, one generator per problem."""
    sizes = []
    for k in range(n_prob):
        rng = np.random.default_rng([seed, k])
        sizes.append(int(np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi))))))
    return sizes


def batched_stokes(sizes, seed: int = 3, dtype=np.float32):
    """Concatenated uniform Stokes problems; problem k uses default_rng([seed, k, 1]).

    Returns (points [sum,3], forces [sum,3], offsets [n_prob+1]).
    """
    pts, fs = [], []
    for k, nk in enumerate(sizes):
        rng = np.random.default_rng([seed, k, 1])
        pts.append(rng.random((nk, 3)))
        fs.append(rng.standard_normal((nk, 3)))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return (_clip_unit(_cast(np.concatenate(pts), dtype)), _cast(np.concatenate(fs), dtype),
            off)


def lognormal_points(n: int, seed: int = 5, m: float = -1.0, s: float = 0.5):
    """Fractional part of log-normal variates, per coordinate (paper Eq. ptdist)."""
    rng = np.random.default_rng(seed)
    u = rng.lognormal(mean=m, sigma=s, size=(n, 3))
    return _clip_unit(u - np.floor(u))


def sample_targets(n: int, k: int = 4096, seed: int = 12345) -> np.ndarray:
    """Sorted indices of k distinct targets (all of them when n <= k)."""
    if n <= k:
        return np.arange(n, dtype=np.int64)
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, k, replace=False)).astype(np.int64)


# The five workloads the evaluator is measured on, with sizes and tree parameters.
WORKLOADS = {
    "laplace_uniform_4k": dict(kernel="laplace", n=4096, p=8, q=64, bc="open"),
    "stokeslet_uniform_256k": dict(kernel="stokeslet", n=262144, p=10, q=128, bc="open"),
    "rpy_clusters_1m": dict(kernel="rpy", n=1048576, p=8, q=128, bc="open"),
    "stokeslet_batched_512": dict(kernel="stokeslet", n_prob=512, p=8, q=64, bc="open"),
    "stokeslet_periodic_4m": dict(kernel="stokeslet", n=4194304, p=12, q=128, bc="pxyz"),
}
