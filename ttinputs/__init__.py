"""Seeded synthetic TT inputs shared by the CPU oracle tests, the GPU parity
tests and the benchmark.

This module only draws random numbers and lays them out as TT cores
(``core[k]`` has shape ``(r_{k-1}, n_k, r_k)`` with ``r_0 = r_d = 1``, the
TT format of Section 2).  It holds none of the method's arithmetic: no sums,
dots, QR, SVD or rounding.  Every generator takes an explicit seed and uses
``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "random_tt",
    "random_tts",
    "coefficients",
    "cfg_mgs_small",
    "cfg_round_sum",
    "cfg_orth_recursive",
    "cfg_batched",
    "cfg_serving_request",
    "rank_profile",
]


def rank_profile(d, n, r):
    """Uniform target rank r capped by the mode products on each side,
    r_k = min(r, prod n_1..n_k, prod n_{k+1}..n_d) with r_0 = r_d = 1."""
    n = [int(v) for v in (n if np.ndim(n) else [n] * d)]
    ranks = [1]
    for k in range(1, d):
        left = int(np.prod(n[:k], dtype=np.float64)) if k <= 40 else 10**18
        right = int(np.prod(n[k:], dtype=np.float64)) if d - k <= 40 else 10**18
        ranks.append(int(min(r, left, right)))
    ranks.append(1)
    return n, ranks


def random_tt(rng, n, ranks, scale=None):
    """iid N(0,1) cores with the given mode sizes and ranks.

    scale: None (plain N(0,1)), or "unit-core" to divide core k by
    sqrt(r_{k-1} n_k) so that entries of the full tensor stay O(1) at any d.
    """
    d = len(n)
    cores = []
    for k in range(d):
        c = rng.standard_normal((ranks[k], n[k], ranks[k + 1]))
        if scale == "unit-core":
            c /= np.sqrt(ranks[k] * n[k])
        cores.append(c)
    return cores


def random_tts(seed, m, d, n, r, scale=None):
    rng = np.random.default_rng(seed)
    nn, ranks = rank_profile(d, n, r)
    return [random_tt(rng, nn, ranks, scale) for _ in range(m)]


def coefficients(seed, m, low=-1.0, high=1.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(low, high, size=m)


def cfg_mgs_small(seed=0, m=10, d=4, n=8, r=4):
    """m TT tensors, order d, mode size n, all ranks r, N(0,1) cores.

    The unit-TT-norm normalisation asked for by this workload is applied by
    the caller with its own TT norm (the generator holds no TT arithmetic);
    ``cfg_mgs_small`` returns raw cores.
    """
    return random_tts(seed, m, d, n, r)


def cfg_round_sum(seed=0, m=20, d=10, n=64, r=20):
    """Inputs of the single-rounding workload: m random TTs (order d, mode n,
    ranks r, N(0,1) cores) and coefficients alpha ~ U(-1, 1)."""
    xs = random_tts(seed, m, d, n, r)
    alpha = coefficients(seed + 7919, m)
    return alpha, xs


def cfg_orth_recursive(seed=0, m=50, d=8, n=32, r=10):
    """Fresh rank-r Gaussian TTs f_1..f_m for the recursive family
    a_k = c a_{k-1} + (1 - c) f_k; the recursion itself (a TT sum) is formed
    by the caller with the code under test."""
    return random_tts(seed, m, d, n, r)


def cfg_batched(seed=0, count=512, d_range=(4, 12), n_choices=(16, 32, 64, 128),
                r_range=(8, 256), max_bytes=None):
    """count independent instances: d ~ U{d_range}, n from n_choices, one
    target rank r ~ U{r_range} per instance (capped by mode products), cores
    N(0,1) divided by sqrt(r_{k-1} n_k) so that no instance overflows fp32."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        n = int(rng.choice(n_choices))
        r = int(rng.integers(r_range[0], r_range[1] + 1))
        nn, ranks = rank_profile(d, n, r)
        out.append(random_tt(rng, nn, ranks, scale="unit-core"))
    return out


def cfg_serving_request(rng, k_range=(1, 64), d_range=(6, 12), n_choices=(32, 64),
                        r_range=(10, 60), deltas=(1e-5, 1e-7)):
    """One request of the serving workload: basis size k, order d, mode n,
    rank r of the new tensor, accuracy delta and its cores."""
    k = int(rng.integers(k_range[0], k_range[1] + 1))
    d = int(rng.integers(d_range[0], d_range[1] + 1))
    n = int(rng.choice(n_choices))
    r = int(rng.integers(r_range[0], r_range[1] + 1))
    delta = float(rng.choice(deltas))
    nn, ranks = rank_profile(d, n, r)
    return dict(k=k, d=d, n=n, r=r, delta=delta,
                cores=random_tt(rng, nn, ranks, scale="unit-core"))
