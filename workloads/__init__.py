"""Seeded synthetic input generators shared by the oracle side and the CUDA side.

This module holds no H²-matrix arithmetic: it only draws point clouds and
right-hand sides.  The point clouds stand in for the centroids of the
triangulated unit sphere the paper uses as its test geometry (Sec. 3.1 and
Sec. 5.1.1); the right-hand sides follow the paper's protocol of random
columns (Sec. 5.1.1).  All generators use numpy's PCG64 ``default_rng`` so a
seed fixes the bytes on any platform.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "sphere_points",
    "ellipsoid_points",
    "gaussian_rhs",
    "batch_specs",
    "CONFIGS",
]


def sphere_points(n: int, seed: int = 0) -> np.ndarray:
    """n points uniform on the unit sphere S² (normalised N(0, I₃) draws), float64 (n, 3)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, 3))
    r = np.sqrt(g[:, 0] * g[:, 0] + g[:, 1] * g[:, 1] + g[:, 2] * g[:, 2])
    return np.ascontiguousarray(g / r[:, None])


def ellipsoid_points(n: int, axes, seed: int = 0) -> np.ndarray:
    """n points on the ellipsoid with semi-axes ``axes``: sphere points scaled per axis."""
    p = sphere_points(n, seed)
    return np.ascontiguousarray(p * np.asarray(axes, dtype=np.float64)[None, :])


def gaussian_rhs(n: int, m: int, seed: int = 1) -> np.ndarray:
    """n×m right-hand sides with i.i.d. N(0, 1) entries, row-major float64."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((n, m)))


def batch_specs(count: int = 64, seed: int = 7, n_lo: int = 2048, n_hi: int = 32768):
    """Specs of independent systems for the batched workload.

    Semi-axes uniform in [0.5, 2], n log-uniform in [n_lo, n_hi], m uniform in
    {1..64}, q uniform in {3, 4}; each system gets its own point and RHS seed.
    """
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        axes = rng.uniform(0.5, 2.0, size=3)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        m = int(rng.integers(1, 65))
        q = int(rng.integers(3, 5))
        specs.append(dict(index=i, n=n, m=m, q=q, axes=tuple(float(a) for a in axes),
                          point_seed=1000 + i, rhs_seed=2000 + i))
    return specs


#: The five workloads: sphere/ellipsoid clouds, kernel exp(-r/0.5) + 1e-2·I,
#: leaf size 64, eta = 2.
CONFIGS = {
    "fp64_n4096": dict(n=4096, q=3, m=8, leaf=64, eta=2.0, length=0.5, sigma=1e-2,
                       point_seed=0, rhs_seed=1),
    "precision_n65536": dict(n=65536, q=4, m=32, leaf=64, eta=2.0, length=0.5, sigma=1e-2,
                             point_seed=0, rhs_seed=1),
    "diff_n262144": dict(n=262144, q=4, m=16, leaf=64, eta=2.0, length=0.5, sigma=1e-2,
                         point_seed=0, rhs_seed=1),
    "scale_n1048576": dict(n=1048576, q=4, m=64, leaf=64, eta=2.0, length=0.5, sigma=1e-2,
                           point_seed=0, rhs_seed=1),
}
