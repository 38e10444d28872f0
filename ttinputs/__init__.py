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


def orthonormal_basis(rng, n, k, rb):
    """k TT tensors with modes n (len(n) >= 3), orthonormal by construction:
    q_(a,b) = u_a (x) v_b (x) w_(a,b), u_a and v_b columns of random
    orthogonal matrices over modes 1 and 2 (k <= n_1 n_2), w a TT over modes
    3..d of rank rb whose cores have orthonormal left unfoldings and whose
    last core is a unit vector, so ||w|| = 1 and <q_i, q_j> = delta_ij.
    TT ranks of each q: [1, 1, 1, rb, ..., rb, 1]."""
    d = len(n)
    if d < 3 or k > n[0] * n[1]:
        raise ValueError("need d >= 3 and k <= n_1 n_2")
    U = np.linalg.qr(rng.standard_normal((n[0], n[0])))[0]
    V = np.linalg.qr(rng.standard_normal((n[1], n[1])))[0]
    out = []
    for j in range(k):
        a, b = j % n[0], j // n[0]
        cores = [U[:, a].reshape(1, n[0], 1), V[:, b].reshape(1, n[1], 1)]
        _, ranks = rank_profile(d - 2, n[2:], rb)
        for m in range(2, d):
            rl, rr = ranks[m - 2], ranks[m - 1]
            M = rng.standard_normal((rl * n[m], rr))
            Qm = np.linalg.qr(M)[0] if m < d - 1 else M / np.linalg.norm(M)
            cores.append(Qm.reshape(rl, n[m], rr))
        out.append(cores)
    return out


def cfg_serving(seed=0, count=256, k_range=(1, 64), d_range=(6, 12), n_choices=(32, 64),
                r_range=(10, 60), deltas=(1e-5, 1e-7), basis_rank=4, orth_fraction=0.5):
    """The serving workload: resident bases, one per (d, n) pair, of
    k_range[1] orthonormal vectors (orthonormal_basis, rank basis_rank), and
    count requests: with probability orth_fraction an orthogonalization step
    of a new rank-r tensor against the first k vectors of the basis of its
    (d, n), else a rounding of a rank-r tensor with graded bonds (columns
    of each core scaled over eight decades, so that delta truncates).  Returns (bases: {(d, n): cores list}, requests: list of dicts
    with kind, d, n, r, k, delta, scheme, cores)."""
    rng = np.random.default_rng(seed)
    bases = {}
    reqs = []
    for _ in range(count):
        q = cfg_serving_request(rng, k_range, d_range, n_choices, r_range, deltas)
        key = (q["d"], q["n"])
        if key not in bases:
            bases[key] = orthonormal_basis(np.random.default_rng([seed, q["d"], q["n"]]),
                                           [q["n"]] * q["d"], k_range[1], basis_rank)
        if rng.random() < orth_fraction:
            q["kind"] = "orth"
            q["scheme"] = str(rng.choice(["cgs2", "mgs2"]))
        else:
            q["kind"] = "round"
            # graded bonds: the j-th column of every core scaled by
            # 10^(-8 j / r), so the bond singular values spread over about
            # eight decades and the rounding at delta truncates them
            for c in q["cores"][:-1]:
                c *= 10.0 ** (-8.0 * np.arange(c.shape[2]) / max(c.shape[2], 1))
            q["scheme"] = None
            q["k"] = 0
        reqs.append(q)
    return bases, reqs

