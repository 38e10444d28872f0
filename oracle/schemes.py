"""The six TT orthogonalization schemes of Section 3, literal, in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every scheme takes a list of TTs A = [a_1..a_m] and an accuracy delta, and
returns (Q, R, n_rounds): the list of TT basis vectors, the m x m upper
triangular R (column i holds the coefficients of a_i) and the number of
TT-round calls made.

Rounding policy:
  "paper"         rounds exactly where Algorithms 1-5 and 8 round;
  "every_update"  rounds p after every axpy of the Gram-Schmidt loops (and,
                  for Householder, every reflected a_j); where a loop makes
                  no update the single rounding of the paper policy is kept.
"""
from __future__ import annotations

import math

import numpy as np

from .tt import canonical_e, tt_add, tt_dot, tt_norm, tt_round, tt_scale

SCHEMES = ("cgs", "mgs", "cgs2", "mgs2", "gram", "householder")


class BreakdownError(ArithmeticError):
    """A zero vector where the scheme normalises (||p|| = 0 or ||w|| = 0)."""


class _Counter:
    def __init__(self, delta):
        self.delta = delta
        self.n = 0

    def round(self, x):
        self.n += 1
        return tt_round(x, self.delta)


def _axpy(p, alpha, q):
    """p + alpha q as a TT concatenation (rank r_p + r_q, Section 2)."""
    return tt_add([1.0, alpha], [p, q])


def _normalize(p):
    nrm = tt_norm(p)
    if nrm == 0.0:
        raise BreakdownError("zero vector in normalisation")
    return nrm, tt_scale(p, 1.0 / nrm)


def _gs(A, delta, policy, modified):
    """Algorithm 1 (TT-CGS, modified=False) and Algorithm 2 (TT-MGS)."""
    m = len(A)
    R = np.zeros((m, m))
    Q = []
    cnt = _Counter(delta)
    for i in range(m):
        p = A[i]
        for j in range(i):
            # reading: the projection is stored at (j, i) so that R is upper
            # triangular with column i belonging to a_i
            R[j, i] = tt_dot(p if modified else A[i], Q[j])
            p = _axpy(p, -R[j, i], Q[j])
            if policy == "every_update":
                p = cnt.round(p)
        if policy == "paper" or i == 0:
            p = cnt.round(p)
        R[i, i], q = _normalize(p)
        Q.append(q)
    return Q, R, cnt.n


def tt_cgs(A, delta, policy="paper"):
    """Algorithm 1, TT-CGS: projections of a_i on q_1..q_{i-1}, one rounding
    per i, R(i,i) = ||p||, q_i = p / R(i,i)."""
    return _gs(A, delta, policy, modified=False)


def tt_mgs(A, delta, policy="paper"):
    """Algorithm 2, TT-MGS: projections of the running p."""
    return _gs(A, delta, policy, modified=True)


def _gs2(A, delta, policy, modified):
    """Algorithm 3 (TT-CGS2) and Algorithm 4 (TT-MGS2): the projection loop
    twice, each followed by a rounding; R = R_1 + R_2."""
    m = len(A)
    R1 = np.zeros((m, m))
    R2 = np.zeros((m, m))
    Q = []
    cnt = _Counter(delta)
    for i in range(m):
        p_prev = A[i]
        for k, Rk in enumerate((R1, R2)):
            p = p_prev
            for j in range(i):
                Rk[j, i] = tt_dot(p if modified else p_prev, Q[j])
                p = _axpy(p, -Rk[j, i], Q[j])
                if policy == "every_update":
                    p = cnt.round(p)
            if policy == "paper" or i == 0:
                p = cnt.round(p)
            p_prev = p
        R2[i, i], q = _normalize(p_prev)
        Q.append(q)
    return Q, R1 + R2, cnt.n


def tt_cgs2(A, delta, policy="paper"):
    """Algorithm 3, TT-CGS2."""
    return _gs2(A, delta, policy, modified=False)


def tt_mgs2(A, delta, policy="paper"):
    """Algorithm 4, TT-MGS2."""
    return _gs2(A, delta, policy, modified=True)


def tt_gram(A, delta, policy="paper"):
    """Algorithm 5, TT-Gram: G(i,j) = <a_i, a_j>, G = L L^T, R = L^T, explicit
    R^{-1} (remark on back-substitution), q_i = sum_{k<=i} R^{-1}(k,i) a_k
    (reading: the equation's index order, R^{-1} upper triangular), one
    rounding per i.  Raises numpy.linalg.LinAlgError when G is not
    numerically SPD (remark on the Gram breakdown)."""
    m = len(A)
    G = np.zeros((m, m))
    for i in range(m):
        for j in range(i + 1):
            G[i, j] = G[j, i] = tt_dot(A[i], A[j])
    L = np.linalg.cholesky(G)
    R = L.T.copy()
    Rinv = np.linalg.inv(R)
    Q = []
    cnt = _Counter(delta)
    for i in range(m):
        p = tt_scale(A[0], Rinv[0, i])
        for j in range(1, i + 1):
            p = _axpy(p, Rinv[j, i], A[j])
            if policy == "every_update":
                p = cnt.round(p)
        if policy == "paper" or i == 0:
            p = cnt.round(p)
        Q.append(p)
    return Q, R, cnt.n


def apply_h_vec(a, u):
    """Algorithm 7: b = a - 2 <a, u> u (no rounding)."""
    return _axpy(a, -2.0 * tt_dot(a, u), u)


def tth_vec(a, F, delta, sign_rule="stable", counter=None):
    """Algorithm 6, TTH-vec: Householder TT-vector u and the column r of R for
    the TT-vector a and canonical vectors F = [f_1..f_i].

    r(j) = <a, f_j> for j < i; w = a - sum_j r(j) f_j, rounded;
    r(i) = s_i sqrt(||a||^2 - sum_j r(j)^2) (clamped at 0, reading of the
    delta-perturbed case); w = w - r(i) f_i, rounded; u = w / ||w|| (reading:
    the listing's ||z|| is ||w||).

    sign_rule "stable": s_i = -sign(<a, f_i>), the cancellation-free choice
    that Section 3.3 attributes to the matrix case; "literal": s_i =
    +sign(<a, f_i>) as printed in the listing.  sign(0) = +1.
    """
    if counter is None:
        counter = _Counter(delta)
    i = len(F)
    r = np.zeros(i)
    s = 0.0
    w = a
    for j in range(i - 1):
        r[j] = tt_dot(a, F[j])
        s += r[j] ** 2
        w = _axpy(w, -r[j], F[j])
    w = counter.round(w)
    t = tt_norm(a) ** 2 - s
    if t < 0.0:
        t = 0.0
    fi = tt_dot(a, F[i - 1])
    sg = 1.0 if fi >= 0.0 else -1.0
    if sign_rule == "stable":
        r[i - 1] = -sg * math.sqrt(t)
    elif sign_rule == "literal":
        r[i - 1] = sg * math.sqrt(t)
    else:
        raise ValueError(sign_rule)
    w = _axpy(w, -r[i - 1], F[i - 1])
    w = counter.round(w)
    _, u = _normalize(w)
    return u, r


def tt_householder(A, delta, policy="paper", sign_rule="stable", return_u=False):
    """Algorithm 8, TT-Householder.

    w = a_1 rounded (reading: one rounding for every a~_k, k = 1..m, which
    gives the 4m roundings of the cost table); for i = 1..m: u_i, R(:i, i) =
    TTH-vec(w, {e_1..e_i}); a_j <- H_i a_j for j = i..m (unrounded under the
    paper policy); w = round(a_{i+1}).  Then q_i = H_1 ... H_i e_i, rounded.
    """
    m = len(A)
    n = [c.shape[1] for c in A[0]]
    if int(np.prod(n, dtype=np.float64)) < m:
        raise ValueError("prod(n) must be >= m for the canonical basis")
    E = [canonical_e(j + 1, n) for j in range(m)]
    R = np.zeros((m, m))
    cnt = _Counter(delta)
    A = list(A)
    U = []
    w = cnt.round(A[0])
    for i in range(m):
        u, r = tth_vec(w, E[: i + 1], delta, sign_rule, cnt)
        R[: i + 1, i] = r
        U.append(u)
        for j in range(i, m):
            A[j] = apply_h_vec(A[j], u)
            if policy == "every_update" and j > i:
                A[j] = cnt.round(A[j])
        if i < m - 1:
            w = cnt.round(A[i + 1])
    Q = []
    for i in range(m):
        q = E[i]
        for j in range(i, -1, -1):
            q = apply_h_vec(q, U[j])
        Q.append(cnt.round(q))
    if return_u:
        return Q, R, cnt.n, U
    return Q, R, cnt.n


def gs_step(a, Q, delta, scheme="cgs2", policy="paper"):
    """One outer iteration of Algorithms 1-4 for the vector a against the
    orthonormal list Q (the step an Arnoldi-type caller issues per new
    vector): the projection loop (once for CGS/MGS, twice for CGS2/MGS2),
    rounding as the policy says, then normalisation.  Returns (q, col, n)
    with col[j] = R(j, i) for j < i = len(Q) (both passes summed), col[i] =
    ||p|| and n the number of roundings."""
    modified = scheme in ("mgs", "mgs2")
    passes = 2 if scheme in ("cgs2", "mgs2") else 1
    i = len(Q)
    col = np.zeros(i + 1)
    cnt = _Counter(delta)
    p_prev = a
    for _ in range(passes):
        p = p_prev
        rk = np.zeros(i)
        for j in range(i):
            rk[j] = tt_dot(p if modified else p_prev, Q[j])
            p = _axpy(p, -rk[j], Q[j])
            if policy == "every_update":
                p = cnt.round(p)
        if policy == "paper" or i == 0:
            p = cnt.round(p)
        col[:i] += rk
        p_prev = p
    col[i], q = _normalize(p_prev)
    return q, col, cnt.n


def loss_of_orthogonality(Q):
    """||I - Q^T Q||_2 with (Q^T Q)(i,j) = <q_i, q_j> from TT dots
    (Section 3.4, eq. LOO; Section 4.1)."""
    m = len(Q)
    G = np.zeros((m, m))
    for i in range(m):
        for j in range(i + 1):
            G[i, j] = G[j, i] = tt_dot(Q[i], Q[j])
    ev = np.linalg.eigvalsh(np.eye(m) - G)
    return float(np.max(np.abs(ev)))


_DISPATCH = {
    "cgs": tt_cgs,
    "mgs": tt_mgs,
    "cgs2": tt_cgs2,
    "mgs2": tt_mgs2,
    "gram": tt_gram,
    "householder": tt_householder,
}


def orthogonalize(scheme, A, delta, policy="paper", **kw):
    return _DISPATCH[scheme](A, delta, policy, **kw)
