"""Seeded synthetic inputs: degree / weight sequences sorted non-increasing.

This module holds none of the sampler's arithmetic; it only produces the
weight sequences that both the CUDA path and the CPU oracle consume.  The
paper's real networks (Miami, Twitter, Friendster; Table 1) are not
available, so discrete power laws and constant (Erdos-Renyi) weights stand in
for its PL and ER rows.

A sorted i.i.d. sample from a discrete distribution has the same law as the
expansion of a multinomial count vector over the support, which is how the
sequences are drawn (one multinomial draw instead of n inverse-CDF draws and
a sort).
"""
from __future__ import annotations

import math

import numpy as np


def powerlaw_pmf(gamma: float, dmin: int, dmax: int):
    d = np.arange(dmin, dmax + 1, dtype=np.float64)
    p = d ** (-gamma)
    return d.astype(np.int64), p / p.sum()


def powerlaw_degrees(n: int, gamma: float, dmin: int, dmax: int, seed: int) -> np.ndarray:
    """n i.i.d. degrees with P(d) proportional to d^-gamma on [dmin, dmax], sorted
    non-increasing, as int32."""
    vals, pmf = powerlaw_pmf(gamma, dmin, dmax)
    rng = np.random.default_rng(seed)
    counts = rng.multinomial(n, pmf)
    return np.repeat(vals[::-1].astype(np.int32), counts[::-1])


def constant_weights(n: int, c: int) -> np.ndarray:
    """Erdos-Renyi special case: w_u = c for every node, so p = c / n."""
    return np.full(n, c, dtype=np.int32)


# Named workloads (sizes and distributions of the paper's PL/ER experiments,
# scaled to one GPU).
def workload(name: str):
    """Returns (weights, edge_seed) for a named workload."""
    if name == "pl_n1e5":  # gamma 2.5 on [2, 1000], degree seed 1
        return powerlaw_degrees(100_000, 2.5, 2, 1000, 1), 42
    if name == "pl_n1e7":  # gamma 2.5 on [10, 10^4], degree seed 2
        return powerlaw_degrees(10_000_000, 2.5, 10, 10_000, 2), 42
    if name == "pl_n1e8":  # gamma 2.3 on [20, 10^5], degree seed 3
        return powerlaw_degrees(100_000_000, 2.3, 20, 100_000, 3), 42
    if name == "er_n1e8":  # w = 100 everywhere
        return constant_weights(100_000_000, 100), 42
    raise KeyError(name)


def batch_graph_params(g: int):
    """Graph g of the batched workload: n log-uniform in [10^3, 10^6], gamma
    uniform in [2.1, 3.0], degrees on [2, floor(sqrt(n))], seeds from g."""
    rng = np.random.default_rng([g, 0x475052])
    n = int(math.floor(10 ** (3 + 3 * rng.random())))
    gamma = 2.1 + 0.9 * rng.random()
    return n, gamma, 2, max(2, int(math.isqrt(n)))


def batch_workload(G: int = 4096):
    """List of (weights, seed) for G graphs; graph g uses edge seed g."""
    out = []
    for g in range(G):
        n, gamma, a, b = batch_graph_params(g)
        out.append((powerlaw_degrees(n, gamma, a, b, g + 1_000_000), g))
    return out


def calibration_targets(n: int = 10_000_000, seed: int = 5) -> np.ndarray:
    """Target degrees for weight calibration: gamma 2.1 on [5, 2*10^5], float64."""
    return powerlaw_degrees(n, 2.1, 5, 200_000, seed).astype(np.float64)
