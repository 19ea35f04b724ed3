"""Seeded synthetic workloads shaped like the paper's datasets.

This module holds random-number recipes only (no join arithmetic); both the
CUDA path's tests/benchmark and the CPU oracle's tests draw their inputs from
it.  Every generator is a pure function of its arguments and seed.

Workloads (sizes from the paper's dataset table, Tab. datasets, and the
project's benchmark configurations):

* ``gauss_small``   X 10,000 x 32, 16-component isotropic Gaussian mixture
                    (centres ~ N(0, 4I), sigma 1); 5 % of the 1,000 queries are
                    drawn from the same mixture shifted by 8 along a seeded unit
                    vector (out of distribution).
* ``sift_like``     X 1,000,000 x 128 integers 0..255 stored as float32: 256
                    centres ~ U[32, 224]^d, points round(clip(mu + N(0, 20^2 I),
                    0, 255)); 100,000 queries, 90 % from the same mixture, 10 %
                    from 256 fresh centres shifted by +64 (then clipped).
                    ``scale`` shrinks both counts (same recipe) for tests.
* ``angular_instance`` / ``angular_collection``
                    a collection of independent join instances of very
                    different sizes (the scalability study's shape): |X|
                    log-uniform in [1e4, 2e6], |Q| log-uniform in [1e3, 2e5]
                    clipped to |X|, d = 100 unit vectors (cosine), 64 clusters
                    per instance (centres uniform on the sphere, points
                    normalise(mu + N(0, 0.07^2 I))), 10 % of the queries from 64
                    fresh centres; a target of U{5..50} matches per query.
                    The size ranges are parameters, so tests draw small
                    collections from the same recipe.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Workload:
    name: str
    X: np.ndarray          # data vectors  [nx, d] float32
    Q: np.ndarray          # query vectors [nq, d] float32
    ood: np.ndarray        # [nq] bool: query drawn from the shifted mixture
    metric: int            # 0 = L2, 1 = cosine
    degree: int            # graph degree R
    knn_k: int             # kNN candidates per node for the graph build
    target_matches: float  # mean matches per query used to set eps
    seed: int

    @property
    def nx(self):
        return self.X.shape[0]

    @property
    def nq(self):
        return self.Q.shape[0]

    @property
    def d(self):
        return self.X.shape[1]


def _mixture(rng, n, centres, sigma):
    lab = rng.integers(0, centres.shape[0], size=n)
    pts = centres[lab] + rng.standard_normal((n, centres.shape[1]), dtype=np.float32) * np.float32(sigma)
    return pts.astype(np.float32)


def gauss_small(seed: int = 1235, nx: int = 10_000, nq: int = 1_000, d: int = 32, k: int = 16,
                ood_frac: float = 0.05, shift: float = 8.0) -> Workload:
    rng = np.random.default_rng(seed)
    centres = (rng.standard_normal((k, d)) * 2.0).astype(np.float32)
    X = _mixture(rng, nx, centres, 1.0)
    n_ood = int(round(nq * ood_frac))
    Qi = _mixture(rng, nq - n_ood, centres, 1.0)
    e = rng.standard_normal(d)
    e = (e / np.linalg.norm(e)).astype(np.float32)
    Qo = _mixture(rng, n_ood, centres + np.float32(shift) * e, 1.0)
    Q = np.concatenate([Qi, Qo]).astype(np.float32)
    ood = np.zeros(nq, bool)
    ood[nq - n_ood:] = True
    perm = rng.permutation(nq)
    return Workload("gauss_small", X, Q[perm].copy(), ood[perm].copy(), 0, 16, 32, 10.0, seed)


def sift_like(seed: int = 1236, scale: float = 1.0, nx: int = 1_000_000, nq: int = 100_000,
              d: int = 128, k: int = 256, ood_frac: float = 0.10, sigma: float = 20.0,
              shift: float = 64.0) -> Workload:
    nx = max(1, int(round(nx * scale)))
    nq = max(1, int(round(nq * scale)))
    rng = np.random.default_rng(seed)
    centres = rng.uniform(32.0, 224.0, size=(k, d)).astype(np.float32)

    def ints(pts):
        return np.clip(np.rint(pts), 0, 255).astype(np.float32)

    X = ints(_mixture(rng, nx, centres, sigma))
    n_ood = int(round(nq * ood_frac))
    Qi = ints(_mixture(rng, nq - n_ood, centres, sigma))
    fresh = rng.uniform(32.0, 224.0, size=(k, d)).astype(np.float32) + np.float32(shift)
    Qo = ints(_mixture(rng, n_ood, fresh, sigma))
    Q = np.concatenate([Qi, Qo]).astype(np.float32)
    ood = np.zeros(nq, bool)
    ood[nq - n_ood:] = True
    perm = rng.permutation(nq)
    return Workload("sift_like", X, Q[perm].copy(), ood[perm].copy(), 0, 32, 64, 20.0, seed)


def uniform_small(seed: int, nx: int, nq: int, d: int, metric: int = 0, degree: int = 8,
                  knn_k: int = 16) -> Workload:
    """Unstructured small case (uniform cube, or unit sphere for cosine)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((nx, d)).astype(np.float32)
    Q = rng.standard_normal((nq, d)).astype(np.float32)
    if metric == 1:
        X /= np.linalg.norm(X, axis=1, keepdims=True)
        Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    return Workload("uniform_small", X, Q, np.zeros(nq, bool), metric, degree, knn_k, 5.0, seed)


def _unit(a):
    return (a / np.linalg.norm(a, axis=1, keepdims=True)).astype(np.float32)


def angular_instance(seed: int, i: int, nx_range=(1e4, 2e6), nq_range=(1e3, 2e5), d: int = 100,
                     k: int = 64, sigma: float = 0.07, ood_frac: float = 0.10) -> Workload:
    """Instance i of an angular collection (a pure function of seed and i)."""
    rng = np.random.default_rng([seed, i])
    lx = rng.uniform(np.log(nx_range[0]), np.log(nx_range[1]))
    lq = rng.uniform(np.log(nq_range[0]), np.log(nq_range[1]))
    nx = int(round(np.exp(lx)))
    nq = min(int(round(np.exp(lq))), nx)
    target = float(rng.integers(5, 51))
    centres = _unit(rng.standard_normal((k, d)))
    X = _unit(_mixture(rng, nx, centres, sigma))
    n_ood = int(round(nq * ood_frac))
    Qi = _unit(_mixture(rng, nq - n_ood, centres, sigma))
    Qo = _unit(_mixture(rng, n_ood, _unit(rng.standard_normal((k, d))), sigma))
    Q = np.concatenate([Qi, Qo]).astype(np.float32)
    ood = np.zeros(nq, bool)
    ood[nq - n_ood:] = True
    perm = rng.permutation(nq)
    return Workload(f"angular_{i}", X, Q[perm].copy(), ood[perm].copy(), 1, 32, 64, target, seed)


def angular_collection(seed: int = 1239, n: int = 64, **kw):
    """The n instances of an angular collection, generated one at a time."""
    for i in range(n):
        yield angular_instance(seed, i, **kw)
