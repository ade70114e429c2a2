"""Seeded request streams for the serving workload (seed 6).

Poisson arrivals at a given rate, k log-uniform in [k_lo, k_hi], nprobe drawn
uniformly from a small set, query index uniform over the query pool.
"""

from __future__ import annotations

import numpy as np


def request_stream(n: int, rate: float, n_queries: int, seed: int = 6, k_lo: int = 100, k_hi: int = 50_000,
                   nprobes=(32, 128, 512)):
    """Returns (arrival times in seconds from 0, k[n], nprobe[n], query index[n])."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    arr = np.cumsum(gaps) - gaps[0]
    ks = np.floor(np.exp(rng.uniform(np.log(k_lo), np.log(k_hi), size=n))).astype(np.int32)
    ps = rng.choice(np.asarray(nprobes, dtype=np.int32), size=n)
    qi = rng.integers(0, n_queries, size=n)
    return arr, ks, ps, qi
