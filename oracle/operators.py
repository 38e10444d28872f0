"""TT-matrices, the TT matrix-vector product, rank-capped rounding and the
Krylov input family of the paper's experiments (Section 4), in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A TT-matrix (TT-operator) is a list of 4-way cores; ``cores[k]`` has shape
``(R_{k-1}, m_k, n_k, R_k)`` (output index m_k, input index n_k) with
``R_0 = R_d = 1``: M((i_1..i_d), (j_1..j_d)) = M_1(i_1, j_1) ... M_d(i_d, j_d),
each M_k(i_k, j_k) = core_k(:, i_k, j_k, :) an R_{k-1} x R_k matrix, the
operator form of the TT representation of Section 2.
"""
from __future__ import annotations

import math

import numpy as np

from .tt import _truncation_rank, tt_norm, tt_orthogonalize_rl, tt_scale


def laplace_1d(n):
    """The 1-D Dirichlet Laplacian stencil tridiag(-1, 2, -1) of order n
    (the grid scaling is dropped: the experiments normalise every vector)."""
    return 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)


def laplacian_ttm(d, n):
    """TT-matrix of the d-dimensional Dirichlet Laplacian
    Delta_d = sum_k I (x) ... (x) L (x) ... (x) I with L = laplace_1d(n) in
    the k-th factor (the operator of the Krylov process of Section 4; its
    TT form has ranks 2: first core [L  I], interior cores [[I, 0], [L, I]],
    last core [I; L]).  d = 1 gives L itself."""
    L, I = laplace_1d(n), np.eye(n)
    if d == 1:
        return [L.reshape(1, n, n, 1)]
    first = np.zeros((1, n, n, 2))
    first[0, :, :, 0], first[0, :, :, 1] = L, I
    mid = np.zeros((2, n, n, 2))
    mid[0, :, :, 0], mid[1, :, :, 0], mid[1, :, :, 1] = I, L, I
    last = np.zeros((2, n, n, 1))
    last[0, :, :, 0], last[1, :, :, 0] = I, L
    return [first] + [mid.copy() for _ in range(d - 2)] + [last]


def ttm_full(cores):
    """Dense matrix (prod m_k) x (prod n_k) of a TT-matrix, row and column
    multi-indices in the order of the dense tensors of ``tt_full`` (the
    first mode index slowest)."""
    M = np.ones((1, 1, 1))  # (rows, cols, R)
    for c in cores:
        a, m, n, b = c.shape
        M = np.einsum("xya,aijb->xiyjb", M, c).reshape(M.shape[0] * m, M.shape[1] * n, b)
    return M[:, :, 0]


def tt_matvec(op, x):
    """y = M x for a TT-matrix M and a TT-vector x: core k of y is
    y_k((a, p), i, (b, q)) = sum_j M_k(a, i, j, b) x_k(p, j, q), so the
    ranks multiply (R_k r_k; index a slowest)."""
    if len(op) != len(x):
        raise ValueError("tt_matvec: orders differ")
    out = []
    for M, c in zip(op, x):
        a, m, n, b = M.shape
        p, n2, q = c.shape
        if n != n2:
            raise ValueError("tt_matvec: mode sizes differ")
        out.append(np.einsum("aijb,pjq->apibq", M, c).reshape(a * p, m, b * q))
    return out


def tt_round_rank(cores, delta, max_rank):
    """TT-round(x, delta) with every rank also capped at max_rank (the
    rounding of the Krylov process of Section 4, "the accuracy replaced by a
    maximum TT-rank"): right-to-left QR orthogonalization, then left-to-right
    SVDs, each keeping min(max_rank, minimal rank within eps = delta ||x|| /
    sqrt(d - 1)) singular values.  max_rank <= 0: no cap (= tt_round)."""
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
        if max_rank > 0:
            r = min(r, max_rank)
        y[k] = U[:, :r].reshape(a, n, r)
        y[k + 1] = np.tensordot(S[:r, None] * Vt[:r], y[k + 1], axes=(1, 0))
    return y


def ones_tt(n):
    """The all-ones tensor as a rank-1 TT (the Krylov start vector of
    Section 4)."""
    return [np.ones((1, k, 1)) for k in n]


def krylov_inputs(op, x1, m, max_rank=1, delta=0.0):
    """The input family of Section 4: a_j = TT-round(x_j) (rank capped at
    max_rank) normalised, x_{j+1} = -M a_j, for j = 1..m, from the start
    vector x_1.  Returns [a_1, ..., a_m]."""
    A = []
    x = x1
    for _ in range(m):
        y = tt_round_rank(x, delta, max_rank)
        nrm = tt_norm(y)
        if nrm == 0.0:
            raise ArithmeticError("zero Krylov vector")
        a = tt_scale(y, 1.0 / nrm)
        A.append(a)
        x = tt_scale(tt_matvec(op, a), -1.0)
    return A


def loo_curve(Q):
    """LOO_k = ||I_k - Q_k^T Q_k||_2 for the first k vectors, k = 1..m
    (Section 4.1: the loss of orthogonality as the basis grows), from one
    m x m Gram matrix of TT dots."""
    from .tt import tt_dot
    m = len(Q)
    G = np.zeros((m, m))
    for i in range(m):
        for j in range(i + 1):
            G[i, j] = G[j, i] = tt_dot(Q[i], Q[j])
    out = []
    for k in range(1, m + 1):
        ev = np.linalg.eigvalsh(np.eye(k) - G[:k, :k])
        out.append(float(np.max(np.abs(ev))))
    return out
