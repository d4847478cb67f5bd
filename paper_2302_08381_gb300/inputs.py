"""Seeded synthetic point clouds for tests and benchmarks.

This module holds no spherical-harmonics arithmetic; it only draws inputs, so
that the oracle and the CUDA path can be fed identical bytes. Every generator
draws in FP64 from ``numpy.random.default_rng(seed)`` and casts at the end.

The paper (Section 3) times 10,000 and 100,000 points without stating their
distribution; the workloads below fix it.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "normal_points",
    "shell_points",
    "near_pole_points",
    "pole_mix_points",
    "ragged_sets",
    "upstream",
]


def normal_points(n: int, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """[n, 3] i.i.d. standard normal coordinates."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 3)).astype(dtype)


def _directions(rng, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    nrm = np.linalg.norm(v, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return v / nrm


def shell_points(n: int, rmin: float, rmax: float, seed: int = 0, dtype=np.float32) -> np.ndarray:
    """[n, 3] points with uniform directions and radius ~ U[rmin, rmax]."""
    rng = np.random.default_rng(seed)
    d = _directions(rng, n)
    r = rng.uniform(rmin, rmax, size=(n, 1))
    return (d * r).astype(dtype)


def near_pole_points(n: int, max_angle: float = 1e-4, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """[n, 3] unit vectors within ``max_angle`` rad of +z (first half) or -z.

    theta ~ U[0, max_angle], phi ~ U[0, 2 pi); the second half is mirrored to
    theta -> pi - theta.
    """
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, max_angle, size=n)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n)
    sgn = np.where(np.arange(n) < (n + 1) // 2, 1.0, -1.0)
    st = np.sin(th)
    out = np.stack([st * np.cos(ph), st * np.sin(ph), sgn * np.cos(th)], axis=1)
    return out.astype(dtype)


def pole_mix_points(n: int, max_angle: float = 1e-4, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """Half uniform on the unit sphere, half within ``max_angle`` of the poles."""
    rng = np.random.default_rng(seed)
    a = n // 2
    uni = _directions(rng, a)
    pole = near_pole_points(n - a, max_angle, seed=int(rng.integers(1 << 31)), dtype=np.float64)
    return np.concatenate([uni, pole], axis=0).astype(dtype)


def ragged_sets(nsets: int, lmax_choices, nmin: int, nmax: int, seed: int = 0):
    """Sizes log-uniform in [nmin, nmax] and an l_max per set drawn from a list.

    Returns (sizes int64 [nsets], lmax int32 [nsets], xyz float32 [sum sizes, 3]
    standard normal).
    """
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=nsets))).astype(np.int64)
    lmax = rng.choice(np.asarray(lmax_choices, dtype=np.int32), size=nsets)
    xyz = rng.standard_normal((int(sizes.sum()), 3)).astype(np.float32)
    return sizes, lmax.astype(np.int32), xyz


def upstream(n: int, k: int, seed: int = 0, dtype=np.float32) -> np.ndarray:
    """[n, k] i.i.d. standard normal upstream gradient / cotangent."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, k)).astype(dtype)
