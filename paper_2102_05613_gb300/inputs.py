"""Seeded synthetic inputs: couplings, initial spins and workload mixes.

This module holds none of the sampler's arithmetic.  It only draws the random
problem instances (Sherrington-Kirkpatrick couplings J and starting spin
configurations) that the CUDA path, its checks and the benchmark all consume,
so that every side sees byte-identical inputs.

Couplings follow the SK model of Sec. IV.A: a symmetric N x N matrix with a
zero diagonal, J_ij ~ N(0, 1/N) for the Gaussian model (the paper's J/sqrt(L)
normalisation) or J_ij = +-1 equiprobable for the +-J model.
"""
from __future__ import annotations

import math

import numpy as np

PM1 = 0      # +-J couplings, int8
GAUSS = 1    # Gaussian couplings, float32


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def couplings_pm1(N: int, seed: int) -> np.ndarray:
    """Symmetric int8 matrix, J_ij = +-1 equiprobable for i != j, J_ii = 0."""
    bits = _rng(seed).integers(0, 2, size=(N, N), dtype=np.int8)
    upper = np.triu(2 * bits - 1, 1).astype(np.int8)
    return (upper + upper.T).astype(np.int8)


def couplings_gauss(N: int, seed: int) -> np.ndarray:
    """Symmetric float32 matrix, J_ij ~ N(0, 1/N) for i != j, J_ii = 0.

    Drawn in float64 and rounded to float32 once; both the GPU path and the
    oracle read these float32 values."""
    g = _rng(seed).standard_normal((N, N)) / math.sqrt(N)
    upper = np.triu(g, 1)
    return (upper + upper.T).astype(np.float32)


def couplings(N: int, kind: int, seed: int) -> np.ndarray:
    return couplings_pm1(N, seed) if kind == PM1 else couplings_gauss(N, seed)


def initial_spins(chains: int, N: int, seed: int) -> np.ndarray:
    """chains x N int8 spins, +-1 equiprobable (a random start)."""
    bits = _rng(seed).integers(0, 2, size=(chains, N), dtype=np.int8)
    return (1 - 2 * bits).astype(np.int8)


def uneven_batch(n_instances: int = 256, seed: int = 0):
    """Instance mix of uneven sizes: N uniform in 128..4096, half +-J and half
    Gaussian, 256..2048 chains each, K uniform in 16..256, beta uniform in
    [0.5, 3].  Returns a list of dicts (no couplings drawn yet)."""
    r = _rng(seed)
    out = []
    for i in range(n_instances):
        out.append(dict(
            N=int(r.integers(128, 4097)),
            kind=PM1 if i % 2 == 0 else GAUSS,
            chains=2 * int(r.integers(128, 1025)),
            K=int(r.integers(16, 257)),
            beta=float(r.uniform(0.5, 3.0)),
            jseed=1000 + i,
        ))
    return out


def poisson_jobs(rate: float, duration: float, seed: int = 0, n_max: int = 8192,
                 steps_range=(1_000, 100_000), chains_max: int = 4096):
    """Sampling jobs arriving as a Poisson process of the given rate (per
    second): N log-uniform in [64, n_max], +-J or Gaussian with equal odds,
    beta uniform in [0.3, 3], K in {1, 16, 64, 256} (K = 1 is plain
    Metropolis), steps log-uniform in steps_range, chains log-uniform in
    [1, chains_max].  Returns a list of dicts sorted by arrival time."""
    r = _rng(seed)
    t = 0.0
    jobs = []
    while True:
        t += float(r.exponential(1.0 / rate))
        if t >= duration:
            break
        N = int(round(math.exp(r.uniform(math.log(64), math.log(n_max)))))
        K = int(r.choice([1, 16, 64, 256]))
        steps = int(round(math.exp(r.uniform(math.log(steps_range[0]), math.log(steps_range[1])))))
        chains = int(round(math.exp(r.uniform(0.0, math.log(chains_max)))))
        jobs.append(dict(
            t_arrive=t, N=max(N, 2), kind=int(r.integers(0, 2)),
            beta=float(r.uniform(0.3, 3.0)), K=K, steps=steps,
            chains=max(chains, 1), jseed=int(r.integers(0, 2**31)),
            seed=int(r.integers(0, 2**62)),
        ))
    return jobs
