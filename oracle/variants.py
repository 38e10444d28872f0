"""Variants of TT-rounding and of TT-Householder beside the paper's own
algorithms, in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* Randomized TT-rounding (cited in Section 2 for large-scale tensors): the
  randomize-then-orthogonalize sketch of the right parts of x by a random
  TT, then one left-to-right sweep of QR factorizations.
* Gram-SVD TT-rounding: the left-to-right truncation of TT-round computed
  from the Gram matrices of the left and right parts of x at each bond,
  without orthogonalizing the cores first.
* TT-Householder with implicit Q (Sections 4.4 and 5: only the Householder
  TT-vectors u_k are stored; q_j = H_1 ... H_j e_j is formed on demand).
"""
from __future__ import annotations

import math

import numpy as np

from .schemes import apply_h_vec
from .tt import _truncation_rank, canonical_e, tt_norm, tt_round


# ---------------------------------------------------------------- randomized
def right_sketch_contractions(x, omega):
    """W[k] (r_k x l_k) = contraction of the right part of x at bond k
    (cores k..d-1, 0-based) with the right part of the random TT omega:
    W[d] = 1, W[k] = sum_i X_k(i) W[k+1] Omega_k(i)^T."""
    d = len(x)
    W = [None] * (d + 1)
    W[d] = np.ones((1, 1))
    for k in range(d - 1, 0, -1):
        W[k] = np.einsum("aib,bc,dic->ad", x[k], W[k + 1], omega[k])
    return W


def tt_round_randomized(x, omega, delta=0.0):
    """Randomize-then-orthogonalize rounding of x with the random TT omega
    (same modes, ranks l; its entries are the method's random draws, passed
    in): W = right_sketch_contractions(x, omega); for k = 1..d-1, the sketch
    Z = X_k^L W[k] of the current core's left unfolding, Z = Q R (LAPACK
    QR), core k <- Q, core k+1 <- (Q^T X_k^L) core k+1.  The ranks become
    at most l.  delta > 0: the result is then rounded by TT-round(., delta)."""
    d = len(x)
    if d == 1:
        return [x[0].copy()]
    y = [c.copy() for c in x]
    W = right_sketch_contractions(x, omega)
    for k in range(d - 1):
        a, n, b = y[k].shape
        XL = y[k].reshape(a * n, b)
        Z = XL @ W[k + 1]
        Q, _ = np.linalg.qr(Z, mode="reduced")
        l = Q.shape[1]
        M = Q.T @ XL
        y[k] = Q.reshape(a, n, l)
        y[k + 1] = np.tensordot(M, y[k + 1], axes=(1, 0))
    if delta > 0:
        y = tt_round(y, delta)
    return y


# ---------------------------------------------------------------- Gram-SVD
def right_grams(x):
    """G_R[k] (r_k x r_k) = R_k R_k^T for the right part R_k of x at bond k
    (cores k..d-1, 0-based): G_R[d-1] = X_{d-1}^R X_{d-1}^R^T and
    G_R[k] = sum_i X_k(i) G_R[k+1] X_k(i)^T."""
    d = len(x)
    G = [None] * d
    c = x[d - 1]
    G[d - 1] = c.reshape(c.shape[0], -1) @ c.reshape(c.shape[0], -1).T
    for k in range(d - 2, 0, -1):
        G[k] = np.einsum("aib,bc,dic->ad", x[k], G[k + 1], x[k])
    return G


def _psd_factor(G, tol_rel):
    """V diag(sqrt(lam)) and V diag(1/sqrt(lam)) over the eigenpairs of the
    symmetric G with lam > tol_rel * lam_max (a square root and the
    pseudo-inverse of its transpose)."""
    lam, V = np.linalg.eigh(0.5 * (G + G.T))
    lmax = max(lam.max(), 0.0)
    keep = lam > tol_rel * lmax
    lam, V = lam[keep], V[:, keep]
    return V * np.sqrt(lam), V / np.sqrt(lam)


def tt_round_gram_svd(x, delta, max_rank=0):
    """TT-round(x, delta) computed from Gram matrices (no orthogonalization of
    the cores): right Grams G_R by one right-to-left sweep of contractions;
    then, for k = 1..d-1, the left Gram G_L of the current left unfolding
    (the cores to its left are already orthonormal), G_L = A A^T and
    G_R = B B^T (eigen-factors, eigenvalues below r u lam_max dropped), the
    SVD A^T B = U S V^T, the minimal rank r' with discarded tail <= eps =
    delta ||x|| / sqrt(d - 1) (||x|| = ||S||_2 at the first bond; at most
    max_rank if > 0), core k <- core k A^+T U_r', core k+1 <- S_r' V_r'^T
    B^+ core k+1.  Accuracy is limited to about sqrt(r u) ||x|| by the
    squared condition numbers of the Grams."""
    d = len(x)
    if d == 1:
        return [x[0].copy()]
    u = 2.0 ** -53
    y = [c.copy() for c in x]
    GR = right_grams(x)
    eps = None
    for k in range(d - 1):
        a, n, b = y[k].shape
        XL = y[k].reshape(a * n, b)
        GL = XL.T @ XL
        A, Ainv_t = _psd_factor(GL, b * u)
        B, Binv_t = _psd_factor(GR[k + 1], b * u)
        U, S, Vt = np.linalg.svd(A.T @ B, full_matrices=False)
        if eps is None:
            eps = delta * float(np.sqrt(np.sum(S ** 2))) / math.sqrt(d - 1)
        r = _truncation_rank(S, eps)
        if max_rank > 0:
            r = min(r, max_rank)
        y[k] = (XL @ (Ainv_t @ U[:, :r])).reshape(a, n, r)
        y[k + 1] = np.tensordot(S[:r, None] * (Vt[:r] @ Binv_t.T), y[k + 1], axes=(1, 0))
    return y


# ---------------------------------------------------------------- Householder
def householder_apply(U, x, transpose=False, delta=None):
    """Q x = H_1 H_2 ... H_k x (transpose False: H_k first) or Q^T x =
    H_k ... H_1 x (H_1 first) for the Householder TT-vectors U = [u_1..u_k]
    (Algorithm 7 for each reflection); with delta, each reflected vector is
    TT-rounded (the rounding of Algorithm 8's q_j formation happens once, at
    the end, when delta is None there)."""
    order = range(len(U)) if transpose else range(len(U) - 1, -1, -1)
    y = x
    for j in order:
        y = apply_h_vec(y, U[j])
        if delta is not None:
            y = tt_round(y, delta)
    return y


def householder_q(U, j, n, delta):
    """q_j = H_1 ... H_j e_j, rounded once (Algorithm 8's last loop) from the
    stored Householder TT-vectors alone.  j is 1-based."""
    return tt_round(householder_apply(U[:j], canonical_e(j, n)), delta)
