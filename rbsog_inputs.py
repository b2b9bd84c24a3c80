"""Seeded synthetic inputs for the RBSOG path: the only module shared by the
oracle-side tests and the CUDA-side tests and benchmark.

It holds input recipes only -- lattices, charges, velocities, batch and
arrival traces -- and none of the method's arithmetic.  Every generator takes
an explicit seed and uses numpy's PCG64.

Recipe of the primitive 1:1 electrolyte (reduced units, number density 0.5):
  * n = ceil(N^(1/3)) sites per side of a simple-cubic lattice with spacing
    a = L / n, site centres at (i + 1/2) a;
  * when N < n^3 the first N sites of a seeded permutation are used;
  * charges: a seeded permutation of N/2 values +1 and N/2 values -1;
  * jitter: uniform in [-0.2, 0.2] per coordinate, then folded into [0, L);
  * velocities: Maxwell-Boltzmann at temperature T for mass m, net momentum
    removed.
"""
from __future__ import annotations

import math

import numpy as np

# Electrolyte workloads (N, L, P) of the paper-shaped benchmarks.
SMALL = dict(N=1000, L=12.6, P=100)           # 1,000 ions, one force + 10 steps
MEDIUM = dict(N=64000, L=50.4, P=200)         # 64,000 ions, 1,000 NVT steps
LARGE = dict(N=1048576, L=128.0, P=500)       # 1,048,576 ions, P in {100, 500, 2000}


def electrolyte(N: int, L: float, seed: int, jitter: float = 0.2, T: float = 1.0,
                mass: float = 1.0):
    """Return (q[N], x[N,3], v[N,3]) in float64 for a neutral 1:1 electrolyte."""
    if N % 2:
        raise ValueError("N must be even for a 1:1 electrolyte")
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(math.ceil(round(N ** (1.0 / 3.0), 9)))
    while n ** 3 < N:
        n += 1
    a = L / n
    idx = np.arange(n ** 3)
    if N < n ** 3:
        idx = rng.permutation(n ** 3)[:N]
        idx.sort()
    ix, iy, iz = idx % n, (idx // n) % n, idx // (n * n)
    x = (np.stack([ix, iy, iz], axis=1).astype(np.float64) + 0.5) * a
    x += rng.uniform(-jitter, jitter, size=x.shape)
    x = np.mod(x, L)
    x[x >= L] = 0.0
    q = np.concatenate([np.ones(N // 2), -np.ones(N // 2)])
    q = q[rng.permutation(N)]
    v = rng.normal(0.0, math.sqrt(T / mass), size=(N, 3))
    v -= v.mean(axis=0, keepdims=True)
    return q, x, v


def random_neutral(N: int, L: float, seed: int, min_dist: float = 0.0):
    """N random charges +-1 (N even) uniform in a cube, optionally with a
    minimum pair distance enforced by rejection (small N only)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = []
    while len(pts) < N:
        p = rng.uniform(0.0, L, size=3)
        ok = True
        for o in pts:
            d = p - o
            d -= L * np.rint(d / L)
            if np.dot(d, d) < min_dist * min_dist:
                ok = False
                break
        if ok:
            pts.append(p)
    q = np.concatenate([np.ones(N // 2), -np.ones(N // 2)])[rng.permutation(N)]
    return q, np.array(pts)


def replica_sizes(n_sys: int, seed: int, n_min: int = 1000, n_max: int = 100000,
                  density: float = 0.5):
    """Batched-replica recipe: N log-uniform in [n_min, n_max] (rounded to
    even), L = (N / density)^(1/3), Bjerrum length uniform in [0.7, 1.5]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_sys))
    N = (np.round(N / 2) * 2).astype(np.int64)
    L = (N / density) ** (1.0 / 3.0)
    lB = rng.uniform(0.7, 1.5, size=n_sys)
    return N, L, lB


def job_trace(n_jobs: int, seed: int, rate: float = 50.0, n_min: int = 500,
              n_max: int = 200000, steps_min: int = 100, steps_max: int = 10000,
              density: float = 0.5):
    """Serving recipe: Poisson arrivals at `rate` jobs/s, N log-uniform in
    [n_min, n_max] (even), steps uniform in [steps_min, steps_max]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_jobs))
    N = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_jobs))
    N = (np.round(N / 2) * 2).astype(np.int64)
    steps = rng.integers(steps_min, steps_max + 1, size=n_jobs)
    L = (N / density) ** (1.0 / 3.0)
    seeds = rng.integers(1, 2**62, size=n_jobs)
    return [dict(t=float(t[i]), N=int(N[i]), L=float(L[i]), steps=int(steps[i]),
                 seed=int(seeds[i])) for i in range(n_jobs)]
