"""TT primitives of the oracle (plain NumPy float64, CPU).

TEST INFRASTRUCTURE ONLY: imported by tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the product.

A TT tensor is a Python list of cores; ``cores[k]`` has shape
``(r_{k-1}, n_k, r_k)`` with ``r_0 = r_d = 1`` (Section 2, TT representation
x = x_1 x_2 ... x_d, entry x(i_1..i_d) = X_1(i_1) ... X_d(i_d)).
Indices in code are 0-based; the paper's are 1-based.
"""
from __future__ import annotations

import math

import numpy as np


def tt_ranks(cores):
    """TT-ranks (r_0, ..., r_d) of a TT (Section 2)."""
    return [cores[0].shape[0]] + [c.shape[2] for c in cores]


def tt_full(cores):
    """Dense tensor of a TT by contracting the cores left to right
    (Section 2: the TT is the contraction of its d 3-order cores)."""
    out = cores[0].reshape(cores[0].shape[1], cores[0].shape[2])
    for c in cores[1:]:
        a, n, b = c.shape
        out = (out.reshape(-1, a) @ c.reshape(a, n * b)).reshape(-1, b)
    shape = [c.shape[1] for c in cores]
    return out.reshape(shape)


def tt_scale(cores, alpha):
    """alpha * x: scales the last core (any single core would do)."""
    out = [c.copy() for c in cores]
    out[-1] = out[-1] * alpha
    return out


def tt_add(alphas, xs):
    """sum_j alpha_j x_j by rank concatenation (Section 2: the k-th TT-rank of
    x + y is r_k + s_k).

    First core: [alpha_1 X_1^(1) ... alpha_m X_1^(m)] along the right rank.
    Interior cores: block diagonal.  Last core: stacked along the left rank.
    For d = 1 the single core is the plain linear combination.
    """
    m = len(xs)
    if m == 0:
        raise ValueError("tt_add needs at least one term")
    d = len(xs[0])
    for x in xs:
        if len(x) != d or [c.shape[1] for c in x] != [c.shape[1] for c in xs[0]]:
            raise ValueError("tt_add: mode sizes differ")
    if d == 1:
        return [sum(a * x[0] for a, x in zip(alphas, xs))]
    out = []
    # first core
    out.append(np.concatenate([a * x[0] for a, x in zip(alphas, xs)], axis=2))
    # interior cores: block diagonal
    for k in range(1, d - 1):
        ra = sum(x[k].shape[0] for x in xs)
        rb = sum(x[k].shape[2] for x in xs)
        n = xs[0][k].shape[1]
        c = np.zeros((ra, n, rb))
        oa = ob = 0
        for x in xs:
            a, _, b = x[k].shape
            c[oa:oa + a, :, ob:ob + b] = x[k]
            oa += a
            ob += b
        out.append(c)
    # last core: stacked
    out.append(np.concatenate([x[d - 1] for x in xs], axis=0))
    return out


def tt_dot(x, y):
    """Euclidean inner product <x, y> of two TTs by left-to-right contraction:
    W_0 = 1, W_k = sum_i X_k(i)^T W_{k-1} Y_k(i), <x, y> = W_d
    (the TT inner product used throughout Algorithms 1-8)."""
    if len(x) != len(y):
        raise ValueError("tt_dot: orders differ")
    W = np.ones((1, 1))
    for cx, cy in zip(x, y):
        if cx.shape[1] != cy.shape[1]:
            raise ValueError("tt_dot: mode sizes differ")
        W = np.einsum("ab,aic,bid->cd", W, cx, cy)
    return float(W[0, 0])


def tt_orthogonalize_rl(cores):
    """Right-to-left orthogonalization: for k = d..2, Householder QR (LAPACK)
    of the transposed right unfolding, the R factor absorbed into core k-1.
    Returns (cores, ||x||) with cores 2..d right-orthonormal and
    ||x|| = ||core_1||_F.  First half of TT-rounding [Oseledets 2011], which
    Section 2 cites."""
    y = [c.copy() for c in cores]
    d = len(y)
    for k in range(d - 1, 0, -1):
        a, n, b = y[k].shape
        M = y[k].reshape(a, n * b)
        Q, R = np.linalg.qr(M.T, mode="reduced")  # M^T = Q R, Q: (nb x p)
        p = Q.shape[1]
        y[k] = Q.T.reshape(p, n, b)
        # core_{k-1} <- core_{k-1} x_3 R^T
        y[k - 1] = np.tensordot(y[k - 1], R.T, axes=(2, 0))
    return y, float(np.linalg.norm(y[0]))


def tt_norm(cores):
    """||x|| as ||core_1||_F after right-to-left orthogonalization."""
    return tt_orthogonalize_rl(cores)[1]


def _truncation_rank(S, eps):
    """Minimal r >= 1 with sqrt(sum_{j > r} sigma_j^2) <= eps (reading of the
    per-bond rule of TT-rounding; "<=" test, rank never below 1)."""
    S = np.asarray(S, dtype=np.float64)
    tail = np.concatenate([np.cumsum((S[::-1] ** 2))[::-1], [0.0]])  # tail[r]
    eps2 = eps * eps
    for r in range(1, len(S) + 1):
        if tail[r] <= eps2:
            return r
    return max(1, len(S))


def tt_round(cores, delta):
    """TT-round(x, delta) (Section 2): returns x~ with ||x - x~|| <= delta ||x||.

    Right-to-left orthogonalization (QR), then a left-to-right sweep of SVDs
    of the left unfoldings, each truncated to the minimal rank whose discarded
    singular values have root-sum-square <= eps = delta ||x|| / sqrt(d - 1).
    For d = 1 there is no bond and the input is returned unchanged.
    """
    if delta < 0 or not np.isfinite(delta):
        raise ValueError("delta must be finite and >= 0")
    d = len(cores)
    if d == 1:
        return [cores[0].copy()]
    y, nrm = tt_orthogonalize_rl(cores)
    eps = delta * nrm / math.sqrt(d - 1)
    for k in range(d - 1):
        a, n, b = y[k].shape
        U, S, Vt = np.linalg.svd(y[k].reshape(a * n, b), full_matrices=False)
        r = _truncation_rank(S, eps)
        y[k] = U[:, :r].reshape(a, n, r)
        SV = S[:r, None] * Vt[:r]
        y[k + 1] = np.tensordot(SV, y[k + 1], axes=(1, 0))
    return y


def tt_diff_norm(x, y):
    """||x - y|| from the TT of x - y (concatenation with coefficient -1) and
    its right-to-left orthogonalization; avoids the cancellation of
    ||x||^2 + ||y||^2 - 2 <x, y>."""
    return tt_norm(tt_add([1.0, -1.0], [x, y]))


def bond_singular_values(cores):
    """Singular values of every unfolding x_{(k)} (k = 1..d-1), a gauge
    invariant of the tensor: right-to-left orthogonalization, then the
    left-to-right SVD sweep without truncation."""
    d = len(cores)
    y, _ = tt_orthogonalize_rl(cores)
    out = []
    for k in range(d - 1):
        a, n, b = y[k].shape
        U, S, Vt = np.linalg.svd(y[k].reshape(a * n, b), full_matrices=False)
        out.append(S.copy())
        y[k] = U.reshape(a, n, -1)
        y[k + 1] = np.tensordot(S[:, None] * Vt, y[k + 1], axes=(1, 0))
    return out


def canonical_phi(j, n):
    """phi(j) = (i_1, ..., i_d): inverse of psi(i_1..i_d) = i_1 +
    sum_{a>=2} (i_a - 1) m_a with m_a = prod_{b<a} n_b (Section 3.3;
    i_1 runs fastest).  j and the returned indices are 1-based."""
    t = j - 1
    out = []
    for nk in n:
        out.append(t % nk + 1)
        t //= nk
    if t != 0:
        raise ValueError("index beyond prod(n)")
    return tuple(out)


def canonical_e(j, n):
    """Canonical basis TT-vector e_j = e_{i_1} (x) ... (x) e_{i_d} with
    (i_1..i_d) = phi(j): a rank-1 TT (Section 3.3).  j is 1-based."""
    idx = canonical_phi(j, n)
    cores = []
    for nk, ik in zip(n, idx):
        c = np.zeros((1, nk, 1))
        c[0, ik - 1, 0] = 1.0
        cores.append(c)
    return cores


def compression_ratio(cores):
    """Storage in TT format over dense storage, sum r_{i-1} n_i r_i /
    prod n_j (Section 2, eq. comp_ratio)."""
    num = sum(c.shape[0] * c.shape[1] * c.shape[2] for c in cores)
    den = 1.0
    for c in cores:
        den *= c.shape[1]
    return num / den


def compression_gain(x, x_rounded):
    """Ratio of the TT storage before and after rounding (Section 2,
    eq. gain_ratio)."""
    num = sum(c.shape[0] * c.shape[1] * c.shape[2] for c in x)
    den = sum(c.shape[0] * c.shape[1] * c.shape[2] for c in x_rounded)
    return num / den

