"""Seeded synthetic point clouds shaped like the workloads of the paper's experiments.

This module only draws inputs (numpy PCG64, FP64 on the host).  It holds none of the method's
arithmetic, imports nothing from the CUDA path or from the oracle, and is shared by the tests,
the benchmark and the smoke check so that both sides of every comparison see the same arrays.

Distributions:
  * ``uniform``        -- uniform in the unit square (Section 5, third experiment).
  * ``clusters``       -- half uniform in [0,1]^2, half from 8 isotropic Gaussians (sigma 0.01,
                          centres uniform in [0.1,0.9]^2); strengths N(0,1).
  * ``normal``         -- 2D normal N(0.5, 0.15^2) (the batched workload).
  * ``circle``         -- points on the unit circle with N(0, 1e-4^2) jitter.
  * ``rings_plummer``  -- 80% on 20 rings r_k = k/20 with radial N(0, 1e-3^2) spread, 20% from a
                          2D Plummer-like core r = a sqrt(u/(1-u)), a = 0.05, kept when r <= 1.
  * ``disc_uniform`` / ``disc_inv_r`` -- the unit disc uniformly, or with radial density
                          proportional to 1/r (Section 5, Fig. 5.1), total mass 1.
  * ``normal_sq`` / ``layer`` -- N(0, sigma^2) in both coordinates, or x ~ U[0,1] and
                          y ~ N(0, sigma^2), each forced into the unit square by rejection
                          (Section 5, Fig. 5.2 / 5.3).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 10060  # per workload family: 10060 + k


@dataclass
class Cloud:
    x: np.ndarray
    y: np.ndarray
    q: np.ndarray
    name: str


def _rng(seed):
    return np.random.default_rng(seed)


def uniform(n, seed, qdist="uniform"):
    g = _rng(seed)
    x = g.random(n)
    y = g.random(n)
    q = g.uniform(-1.0, 1.0, n) if qdist == "uniform" else g.standard_normal(n)
    return Cloud(x, y, q, "uniform")


def clusters(n, seed, nclusters=8, sigma=0.01):
    g = _rng(seed)
    nu = n // 2
    nc = n - nu
    xu = g.random(nu)
    yu = g.random(nu)
    centres = g.uniform(0.1, 0.9, (nclusters, 2))
    which = np.repeat(np.arange(nclusters), -(-nc // nclusters))[:nc]
    xc = centres[which, 0] + sigma * g.standard_normal(nc)
    yc = centres[which, 1] + sigma * g.standard_normal(nc)
    x = np.concatenate([xu, xc])
    y = np.concatenate([yu, yc])
    order = g.permutation(n)
    q = g.standard_normal(n)
    return Cloud(x[order], y[order], q, "clusters")


def normal(n, seed, mean=0.5, sd=0.15):
    g = _rng(seed)
    x = mean + sd * g.standard_normal(n)
    y = mean + sd * g.standard_normal(n)
    q = g.uniform(-1.0, 1.0, n)
    return Cloud(x, y, q, "normal")


def circle(n, seed, jitter=1e-4):
    g = _rng(seed)
    t = g.uniform(0.0, 2.0 * np.pi, n)
    x = np.cos(t) + jitter * g.standard_normal(n)
    y = np.sin(t) + jitter * g.standard_normal(n)
    q = g.uniform(-1.0, 1.0, n)
    return Cloud(x, y, q, "circle")


def rings_plummer(n, seed, nrings=20, spread=1e-3, core_frac=0.2, a=0.05):
    g = _rng(seed)
    ncore = int(round(core_frac * n))
    nring = n - ncore
    k = np.repeat(np.arange(1, nrings + 1), -(-nring // nrings))[:nring]
    r = k / nrings + spread * g.standard_normal(nring)
    t = g.uniform(0.0, 2.0 * np.pi, nring)
    xr, yr = r * np.cos(t), r * np.sin(t)
    rc = np.empty(0)
    while rc.shape[0] < ncore:
        u = g.random(2 * ncore)
        cand = a * np.sqrt(u / (1.0 - u))
        rc = np.concatenate([rc, cand[cand <= 1.0]])
    rc = rc[:ncore]
    tc = g.uniform(0.0, 2.0 * np.pi, ncore)
    x = np.concatenate([xr, rc * np.cos(tc)])
    y = np.concatenate([yr, rc * np.sin(tc)])
    order = g.permutation(n)
    q = g.random(n)
    return Cloud(x[order], y[order], q, "rings_plummer")


def disc_uniform(n, seed):
    g = _rng(seed)
    r = np.sqrt(g.random(n))
    t = g.uniform(0.0, 2.0 * np.pi, n)
    return Cloud(r * np.cos(t), r * np.sin(t), np.full(n, 1.0 / n), "disc_uniform")


def disc_inv_r(n, seed):
    g = _rng(seed)
    r = g.random(n)  # density ~ 1/r in the plane <=> r uniform in [0, 1]
    t = g.uniform(0.0, 2.0 * np.pi, n)
    return Cloud(r * np.cos(t), r * np.sin(t), np.full(n, 1.0 / n), "disc_inv_r")


def _reject_unit_square(g, n, draw):
    xs, ys = np.empty(0), np.empty(0)
    while xs.shape[0] < n:
        x, y = draw(2 * n)
        keep = (x >= 0) & (x <= 1) & (y >= 0) & (y <= 1)
        xs = np.concatenate([xs, x[keep]])
        ys = np.concatenate([ys, y[keep]])
    return xs[:n], ys[:n]


def normal_sq(n, seed, sigma):
    g = _rng(seed)
    x, y = _reject_unit_square(g, n, lambda m: (sigma * g.standard_normal(m),
                                                sigma * g.standard_normal(m)))
    return Cloud(x, y, g.uniform(-1.0, 1.0, n), "normal_sq")


def layer(n, seed, sigma):
    g = _rng(seed)
    x, y = _reject_unit_square(g, n, lambda m: (g.random(m), sigma * g.standard_normal(m)))
    return Cloud(x, y, g.uniform(-1.0, 1.0, n), "layer")


def sample_targets(n, m, seed):
    """Distinct sample indices for error checks against the direct sum."""
    g = _rng(seed)
    m = min(m, n)
    return np.sort(g.choice(n, size=m, replace=False)).astype(np.int64)


# ---- the named workloads -----------------------------------------------------------------

@dataclass
class Workload:
    name: str
    n: int
    levels: int
    p: int
    theta: float
    n_check: int  # sampled targets for the direct-sum check (0 = all)


PLAIN_FP64 = Workload("uniform N=10240, L=4, theta=1/2, p=17", 10240, 4, 17, 0.5, 0)
MIXED_1M = Workload("clusters N=2^20, L=8, theta=1/2, p=20", 1 << 20, 8, 20, 0.5, 4096)
LARGE_16M = Workload("rings+plummer N=2^24, L=9, theta=1/2, p=30", 1 << 24, 9, 30, 0.5, 2048)


def plain_fp64_cloud():
    return uniform(PLAIN_FP64.n, SEED_BASE + 0)


def mixed_1m_cloud(n=MIXED_1M.n):
    return clusters(n, SEED_BASE + 1)


def large_16m_cloud(n=LARGE_16M.n):
    return rings_plummer(n, SEED_BASE + 4)


def batched_instances(count=512, seed=SEED_BASE + 2, nmin=1e3, nmax=2e5):
    """Instances of the batched workload: N log-uniform in [nmin, nmax], distributions cycling
    uniform square / 2D normal / jittered unit circle, levels so that leaves hold ~32 points."""
    g = _rng(seed)
    ns = np.round(np.exp(g.uniform(np.log(nmin), np.log(nmax), count))).astype(np.int64)
    out = []
    kinds = (uniform, normal, circle)
    for i, n in enumerate(ns):
        c = kinds[i % 3](int(n), seed * 1000 + i)
        L = max(1, int(round(np.log(n / 32.0) / np.log(4.0))))
        while 4 ** L > n:
            L -= 1
        out.append((c, L))
    return out
