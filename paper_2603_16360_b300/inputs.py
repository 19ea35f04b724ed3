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
* ``vmf_like``      X 10,000,000 x 768 unit vectors rounded to BF16 (cosine),
                    a 4,096-component von Mises-Fisher mixture with
                    concentration kappa = 50 (mean directions uniform on the
                    sphere, Wood's rejection sampler for the component along
                    the mean); 1,000,000 queries, 80 % from the same mixture
                    and 20 % from 1,024 unseen mean directions; plus a
                    held-out set of 100,000 queries drawn the same way for
                    training the learned predictor.  ``scale`` shrinks the
                    counts and the number of mixture components together.
* ``gauss_wide``    X = Q = 1,000,000 x 960 float32, a 512-component Gaussian
                    mixture (centres ~ N(0, I), sigma 0.3), the equal-size
                    GIST-shaped precision case.
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
    nh: int = 0            # the last nh rows of Q are held out (training the predictor), not evaluated

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
              shift: float = 64.0, nh: int = 0) -> Workload:
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
    Q, ood = Q[perm].copy(), ood[perm].copy()
    nh = int(round(nh * scale))
    if nh > 0:
        # held-out queries drawn after the evaluated ones, same recipe
        h_ood = rng.random(nh) < ood_frac
        H = np.where(h_ood[:, None], ints(_mixture(rng, nh, fresh, sigma)), ints(_mixture(rng, nh, centres, sigma)))
        Q = np.concatenate([Q, H.astype(np.float32)])
        ood = np.concatenate([ood, h_ood])
    return Workload("sift_like", X, Q, ood, 0, 32, 64, 20.0, seed, nh)


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


def bf16_round(a):
    """Round float32 values to the nearest BF16 value (ties to even), kept as float32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(np.shape(a))


def wood_w(rng, n: int, d: int, kappa: float) -> np.ndarray:
    """Component along the mean direction of n draws from vMF(kappa) on the unit
    sphere of R^d, by Wood's rejection sampler ("Simulation of the von
    Mises Fisher distribution", 1994): a Beta((d-1)/2, (d-1)/2) proposal mapped
    through a Moebius transform, accepted by the log-density test."""
    m = d - 1.0
    b = (-2.0 * kappa + np.sqrt(4.0 * kappa * kappa + m * m)) / m
    x0 = (1.0 - b) / (1.0 + b)
    c = kappa * x0 + m * np.log(1.0 - x0 * x0)
    w = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        z = rng.beta(m / 2.0, m / 2.0, size=todo.size)
        wt = (1.0 - (1.0 + b) * z) / (1.0 - (1.0 - b) * z)
        u = rng.uniform(size=todo.size)
        ok = kappa * wt + m * np.log(1.0 - x0 * wt) - c >= np.log(u)
        w[todo[ok]] = wt[ok]
        todo = todo[~ok]
    return w


def _vmf_rows(rng, mus, lab, w):
    """Unit vectors w * mu + sqrt(1 - w^2) * v, v uniform on the sphere of the
    directions orthogonal to mu (numpy, float64 arithmetic)."""
    mu = mus[lab].astype(np.float64)
    g = rng.standard_normal(mu.shape)
    v = g - (g * mu).sum(1, keepdims=True) * mu
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return (w[:, None] * mu + np.sqrt(np.maximum(1.0 - w * w, 0.0))[:, None] * v).astype(np.float32)


def vmf_like(seed: int = 1238, scale: float = 1.0, nx: int = 10_000_000, nq: int = 1_000_000,
             nh: int = 100_000, d: int = 768, k: int = 4096, k_unseen: int = 1024, kappa: float = 50.0,
             unseen_frac: float = 0.20, device=None) -> Workload:
    """The learned-predictor workload.  Q holds the nq queries followed by the nh
    held-out queries (``ood`` marks queries of unseen components).  With a
    torch CUDA ``device`` the bulk (the Gaussian draws, the projections and the
    BF16 rounding) runs there with a seeded torch generator and X, Q are CUDA
    tensors; the mean directions, labels and Wood draws come from numpy either
    way."""
    nx = max(1, int(round(nx * scale)))
    nq = max(1, int(round(nq * scale)))
    nh = int(round(nh * scale))
    k = max(1, int(round(k * scale)))
    k_unseen = max(1, int(round(k_unseen * scale)))
    rng = np.random.default_rng(seed)
    mus = _unit(rng.standard_normal((k, d)))
    fresh = _unit(rng.standard_normal((k_unseen, d)))
    nqa = nq + nh
    unseen = rng.random(nqa) < unseen_frac
    lab_x = rng.integers(0, k, size=nx)
    lab_q = np.where(unseen, k + rng.integers(0, k_unseen, size=nqa), rng.integers(0, k, size=nqa))
    allmu = np.concatenate([mus, fresh])
    w_x = wood_w(rng, nx, d, kappa)
    w_q = wood_w(rng, nqa, d, kappa)
    if device is None:
        X = bf16_round(_vmf_rows(rng, allmu, lab_x, w_x))
        Q = bf16_round(_vmf_rows(rng, allmu, lab_q, w_q))
    else:
        import torch
        gen = torch.Generator(device=device)
        gen.manual_seed(seed)
        mu_t = torch.from_numpy(allmu).to(device)

        def rows(lab, w):
            out = torch.empty((len(lab), d), dtype=torch.float32, device=device)
            for a in range(0, len(lab), 1 << 20):
                b = min(len(lab), a + (1 << 20))
                mu = mu_t[torch.from_numpy(lab[a:b]).to(device)]
                g = torch.randn((b - a, d), generator=gen, device=device, dtype=torch.float32)
                v = g - (g * mu).sum(1, keepdim=True) * mu
                v = v / v.norm(dim=1, keepdim=True)
                wt = torch.from_numpy(w[a:b]).to(device=device, dtype=torch.float32)[:, None]
                out[a:b] = (wt * mu + torch.sqrt(torch.clamp(1.0 - wt * wt, min=0.0)) * v).to(torch.bfloat16).float()
            return out

        X = rows(lab_x, w_x)
        Q = rows(lab_q, w_q)
    return Workload("vmf_like", X, Q, unseen, 1, 32, 64, 10.0, seed, nh)


def gauss_wide(seed: int = 1237, scale: float = 1.0, nx: int = 1_000_000, nq: int = 1_000_000, d: int = 960,
               k: int = 512, sigma: float = 0.3) -> Workload:
    nx = max(1, int(round(nx * scale)))
    nq = max(1, int(round(nq * scale)))
    rng = np.random.default_rng(seed)
    centres = rng.standard_normal((k, d)).astype(np.float32)
    X = _mixture(rng, nx, centres, sigma)
    Q = _mixture(rng, nq, centres, sigma)
    return Workload("gauss_wide", X, Q, np.zeros(nq, bool), 0, 32, 64, 10.0, seed)
