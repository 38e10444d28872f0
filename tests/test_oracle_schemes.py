"""Pins of the oracle's six orthogonalization schemes (Algorithms 1-8):
  * d = 1 reduces every scheme to its textbook matrix form (TT-round is the
    identity without bonds): compared with LAPACK QR;
  * dense brute force on the small MGS workload (order 4, mode 8, ranks 4);
  * rounding counts of the cost table (golden fixture);
  * rank bounds of Section 4.4.2 for rank-1 inputs;
  * loss-of-orthogonality orders of Section 3.4 / Table tab:orth.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle.schemes import BreakdownError
from ttinputs import random_tt, random_tts

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _as_d1(A):
    return [[A[:, j].reshape(1, -1, 1)] for j in range(A.shape[1])]


def _qr_pos(A):
    Q, R = np.linalg.qr(A)
    s = np.sign(np.diag(R))
    s[s == 0] = 1
    return Q * s, (R.T * s).T


@pytest.mark.parametrize("scheme", ["cgs", "mgs", "cgs2", "mgs2", "gram"])
def test_d1_schemes_equal_matrix_qr(scheme):
    rng = np.random.default_rng(20)
    A = rng.standard_normal((30, 8))
    Q, R, cnt = O.orthogonalize(scheme, _as_d1(A), 0.0)
    Qm = np.column_stack([q[0].ravel() for q in Q])
    Qr, Rr = _qr_pos(A)
    assert np.allclose(Qm, Qr, atol=1e-12)
    assert np.allclose(R, Rr, atol=1e-12)


def test_d1_householder_equals_lapack_householder():
    # LAPACK's dgeqrf uses the same cancellation-free sign rule:
    # R(i,i) = -sign(a~_i(i)) ||a~_i(i:)||, Q = H_1 ... H_m (first m columns)
    rng = np.random.default_rng(21)
    A = rng.standard_normal((25, 7))
    Q, R, cnt = O.tt_householder(_as_d1(A), 0.0)
    Qm = np.column_stack([q[0].ravel() for q in Q])
    Qr, Rr = np.linalg.qr(A)
    assert np.allclose(R, Rr, atol=1e-12)
    assert np.allclose(Qm, Qr, atol=1e-12)
    # literal sign rule: still a valid QR; its first reflection takes the
    # opposite sign (later ones see different reflected vectors)
    Q2, R2, _ = O.tt_householder(_as_d1(A), 0.0, sign_rule="literal")
    Q2m = np.column_stack([q[0].ravel() for q in Q2])
    assert np.allclose(Q2m @ R2, A, atol=1e-9)
    assert np.allclose(Q2m.T @ Q2m, np.eye(7), atol=1e-9)
    assert np.sign(R2[0, 0]) == np.sign(A[0, 0]) == -np.sign(R[0, 0])


def _cfg_small(seed=0, m=10):
    xs = random_tts(seed, m, 4, 8, 4)
    return [O.tt_scale(x, 1.0 / O.tt_norm(x)) for x in xs]


@pytest.mark.parametrize("scheme", ["mgs", "mgs2", "cgs2", "householder", "gram", "cgs"])
@pytest.mark.parametrize("policy", ["paper", "every_update"])
def test_small_workload_dense_brute_force(scheme, policy):
    A = _cfg_small()
    Ad = np.column_stack([O.tt_full(a).ravel() for a in A])  # 4096 x 10
    Q, R, _ = O.orthogonalize(scheme, A, 1e-8, policy)
    Qd = np.column_stack([O.tt_full(q).ravel() for q in Q])
    Qr, Rr = _qr_pos(Ad)
    s = np.sign(np.diag(R))
    assert np.allclose(Qd * s, Qr, atol=1e-6)
    assert np.allclose((R.T * s).T, Rr, atol=1e-6)
    # Q R reproduces A to the rounding accuracy
    assert np.linalg.norm(Qd @ R - Ad) <= 1e-6 * np.linalg.norm(Ad)


def test_rounding_counts_match_cost_table():
    with open(os.path.join(GOLDEN, "tab_orth_rounding_counts.json")) as f:
        per_m = json.load(f)["rounds_per_m"]
    A = _cfg_small(m=6)
    for scheme, c in per_m.items():
        _, _, cnt = O.orthogonalize(scheme, A, 1e-6, "paper")
        assert cnt == c * len(A), scheme


def test_every_update_round_counts():
    m = 5
    A = _cfg_small(m=m)
    gs = sum(max(1, i) for i in range(m))
    assert O.tt_mgs(A, 1e-6, "every_update")[2] == gs
    assert O.tt_cgs(A, 1e-6, "every_update")[2] == gs
    assert O.tt_mgs2(A, 1e-6, "every_update")[2] == 2 * gs
    assert O.tt_gram(A, 1e-6, "every_update")[2] == gs


def _rank1_inputs(seed, m, d, n):
    rng = np.random.default_rng(seed)
    return [random_tt(rng, [n] * d, [1] * (d + 1)) for _ in range(m)]


def test_rank_bounds_for_rank1_inputs():
    # Section 4.4.2: TT-Gram q_k rank <= k, TT-CGS q_k rank <= 1 + k(k-1)/2
    A = _rank1_inputs(30, 6, 4, 5)
    Qg, _, _ = O.tt_gram(A, 1e-10)
    Qc, _, _ = O.tt_cgs(A, 1e-10)
    for k in range(1, 7):
        assert max(O.tt_ranks(Qg[k - 1])) <= k
        assert max(O.tt_ranks(Qc[k - 1])) <= 1 + k * (k - 1) // 2


def test_householder_reflection_is_involution_and_maps_a():
    A = _cfg_small(m=3)
    Q, R, _, U = O.tt_householder(A, 1e-12, return_u=True)
    a = A[1]
    b = O.apply_h_vec(O.apply_h_vec(a, U[0]), U[0])
    assert O.tt_diff_norm(a, b) <= 1e-12
    assert abs(O.tt_norm(U[1]) - 1.0) < 1e-12
    # H_1 a_1 = R(1,1) e_1 up to the rounding accuracy
    n = [c.shape[1] for c in A[0]]
    h = O.apply_h_vec(A[0], U[0])
    e1 = O.canonical_e(1, n)
    assert O.tt_diff_norm(h, O.tt_scale(e1, R[0, 0])) <= 1e-10


def test_gram_breakdown_on_dependent_inputs():
    # an exact repeat makes G exactly singular (remark on the Gram breakdown)
    A = _cfg_small(m=3)
    with pytest.raises(np.linalg.LinAlgError):
        O.tt_gram([A[0], A[1], A[0]], 1e-10)
    with pytest.raises(BreakdownError):
        O.tt_mgs([A[0], O.tt_scale(A[1], 0.0)], 1e-10)


def _ill_conditioned_d1(n, m, kappa, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, m)))
    V, _ = np.linalg.qr(rng.standard_normal((m, m)))
    S = np.logspace(0, -np.log10(kappa), m)
    return (U * S) @ V.T


def test_matrix_loo_orders_at_d1():
    # Section 3.4 with the unit round-off u: CGS ~ u k^2, MGS ~ u k,
    # CGS2 / MGS2 / Householder ~ u.  kappa = 1e6 separates them.
    A = _ill_conditioned_d1(200, 12, 1e6, 22)
    loo = {s: O.loss_of_orthogonality(O.orthogonalize(s, _as_d1(A), 0.0)[0])
           for s in ("cgs", "mgs", "cgs2", "mgs2", "householder")}
    u = 2.0 ** -53
    assert loo["cgs2"] < 1e3 * u and loo["mgs2"] < 1e3 * u and loo["householder"] < 1e3 * u
    assert 1e-2 * u * 1e6 < loo["mgs"] < 1e3 * u * 1e6
    assert loo["cgs"] > 1e2 * loo["mgs"]


def _recursive_family(seed, m, d, n, r, c):
    F = random_tts(seed, m, d, n, r)
    A = [F[0]]
    for k in range(1, m):
        A.append(O.tt_round(O.tt_add([c, 1.0 - c], [A[-1], F[k]]), 1e-14))
    return [O.tt_scale(a, 1.0 / O.tt_norm(a)) for a in A]


def test_tt_loo_orders_in_delta():
    # Table tab:orth, TT column: CGS2 / MGS2 / Householder ~ delta; MGS grows
    # with kappa; CGS and Gram grow with kappa^2 (orders, not constants)
    A = _recursive_family(23, 10, 3, 6, 2, 0.9)
    Ad = np.column_stack([O.tt_full(a).ravel() for a in A])
    kappa = np.linalg.cond(Ad)
    assert kappa > 1e2
    delta = 1e-8
    loo = {s: O.loss_of_orthogonality(O.orthogonalize(s, A, delta)[0]) for s in O.SCHEMES}
    for s in ("cgs2", "mgs2", "householder"):
        assert loo[s] < 1e2 * delta, (s, loo[s])
    assert loo["mgs"] < 1e2 * delta * kappa
    assert loo["cgs"] > loo["mgs2"] and loo["gram"] > loo["mgs2"]


def _conditioned_tt_family(kappa, m=8, n=8, d=3, seed=5):
    # a_i = sum_j M_ji b_j with b_j orthonormal rank-1 TTs (orthonormal factor
    # columns, distinct in the first mode) and M with singular values
    # logspaced from 1 to 1/kappa: the dense matrix [a_1 .. a_m] has
    # condition number kappa exactly
    rng = np.random.default_rng(seed)
    Us = [np.linalg.qr(rng.standard_normal((n, n)))[0] for _ in range(d)]
    perms = [np.arange(m)] + [rng.permutation(m) for _ in range(d - 1)]
    B = [[Us[k][:, perms[k][j]].reshape(1, n, 1) for k in range(d)] for j in range(m)]
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    W = np.linalg.qr(rng.standard_normal((m, m)))[0]
    M = (V * np.logspace(0, -np.log10(kappa), m)) @ W.T
    return [O.tt_add(list(M[:, i]), B) for i in range(m)]


def test_tt_loo_orders_in_kappa():
    # Section 3.4 in TT format with delta far below the round-off effects: the
    # schemes keep their matrix orders in kappa (CGS and Gram ~ u kappa^2,
    # MGS ~ u kappa, CGS2 / MGS2 ~ u; Householder ~ delta).  Growth from
    # kappa = 1e2 to 1e4 is checked, not constants.
    u = 2.0 ** -53
    delta = 1e-10
    loo = {}
    for kappa in (1e2, 1e4):
        A = _conditioned_tt_family(kappa)
        Ad = np.column_stack([O.tt_full(a).ravel() for a in A])
        assert np.linalg.cond(Ad) == pytest.approx(kappa, rel=1e-6)
        loo[kappa] = {s: O.loss_of_orthogonality(O.orthogonalize(s, A, delta)[0]) for s in O.SCHEMES}
    lo, hi = loo[1e2], loo[1e4]
    for s in ("cgs2", "mgs2"):
        assert lo[s] < 1e2 * u and hi[s] < 1e2 * u, (s, lo[s], hi[s])
    assert lo["householder"] < 1e2 * delta and hi["householder"] < 1e2 * delta
    assert 1e1 < hi["mgs"] / lo["mgs"] < 1e3                     # ~ kappa: x 1e2
    assert hi["cgs"] / lo["cgs"] > 1e3 and hi["gram"] / lo["gram"] > 1e3  # ~ kappa^2: x 1e4
    assert hi["cgs"] > 1e2 * hi["mgs"]
    assert 1e-2 * u * 1e4 < hi["mgs"] < 1e2 * u * 1e4


@pytest.mark.parametrize("scheme", ["cgs", "mgs", "cgs2", "mgs2"])
@pytest.mark.parametrize("policy", ["paper", "every_update"])
def test_gs_step_iterated_is_the_scheme(scheme, policy):
    # one outer iteration applied to a_1..a_m in turn is Algorithms 1-4
    A = random_tts(31, 5, 4, 5, 2)
    Q, R, n = O.orthogonalize(scheme, A, 1e-10, policy)
    Qs, nsum = [], 0
    for i, a in enumerate(A):
        q, col, k = O.gs_step(a, Qs, 1e-10, scheme, policy)
        assert np.array_equal(col, R[: i + 1, i])
        for c1, c2 in zip(q, Q[i]):
            assert np.array_equal(c1, c2)
        Qs.append(q)
        nsum += k
    assert nsum == n


@pytest.mark.parametrize("scheme", ["cgs", "mgs", "cgs2", "mgs2"])
def test_gs_step_against_an_orthonormal_basis(scheme):
    # exact orthonormal basis: the coefficients are the projections <a, q_j>,
    # the new vector is a unit vector orthogonal to the basis (up to delta)
    from ttinputs import orthonormal_basis
    rng = np.random.default_rng(32)
    n = [6, 5, 4, 4]
    Q = orthonormal_basis(rng, n, 9, 3)
    G = np.array([[O.tt_dot(a, b) for b in Q] for a in Q])
    assert np.abs(G - np.eye(9)).max() < 1e-13
    a = random_tt(rng, n, [1, 3, 4, 3, 1])
    delta = 1e-10
    q, col, k = O.gs_step(a, Q, delta, scheme)
    proj = np.array([O.tt_dot(a, qj) for qj in Q])
    na = O.tt_norm(a)
    assert np.abs(col[:9] - proj).max() <= 1e-12 * na
    assert k == (2 if scheme.endswith("2") else 1)
    assert abs(O.tt_norm(q) - 1.0) < 1e-12
    assert max(abs(O.tt_dot(q, qj)) for qj in Q) < 10 * delta * na / col[9]
    # dense check: a = sum_j col_j q_j + col_9 q up to the rounding error
    full = sum(c * O.tt_full(v) for c, v in zip(col, Q + [q]))
    assert np.linalg.norm(full - O.tt_full(a)) <= 2 * delta * na


def test_gs_step_first_vector():
    a = random_tts(33, 1, 4, 5, 3)[0]
    q, col, k = O.gs_step(a, [], 1e-3, "mgs2")
    y = O.tt_round(O.tt_round(a, 1e-3), 1e-3)
    assert k == 2 and col.shape == (1,)
    assert col[0] == O.tt_norm(y)
    for c1, c2 in zip(q, O.tt_scale(y, 1.0 / col[0])):
        assert np.array_equal(c1, c2)


def _unit_rank1(rng, n):
    vs = [rng.standard_normal(k) for k in n]
    vs = [v / np.linalg.norm(v) for v in vs]
    return [v.reshape(1, -1, 1) for v in vs]


def test_loss_of_orthogonality_closed_forms():
    # eq. LOO is the spectral norm of I - Q^T Q, with the Gram entries taken
    # from TT dots.  Three sets whose spectral norm is known in closed form
    # and differs from the Frobenius norm, the largest entry and the largest
    # signed eigenvalue, so that any of those mistakes fails:
    rng = np.random.default_rng(77)
    n = [4, 5, 3]
    v = _unit_rank1(rng, n)
    # (a) three copies of one unit vector: I - J_3 has eigenvalues -2, 1, 1,
    #     so the LOO is 2 (Frobenius sqrt(6), largest entry 1, max eig 1)
    assert abs(O.loss_of_orthogonality([v, v, v]) - 2.0) <= 1e-14
    # (b) q_1 = e_1, q_2 = (e_1 + e_2)/sqrt(2): I - G = [[0, -c], [-c, 0]]
    #     with c = 1/sqrt(2); eigenvalues +-c, LOO = c (Frobenius 1)
    e1, e2 = O.canonical_e(1, n), O.canonical_e(2, n)
    q2 = O.tt_scale(O.tt_add([1.0, 1.0], [e1, e2]), 1.0 / np.sqrt(2.0))
    assert abs(O.loss_of_orthogonality([e1, q2]) - 1.0 / np.sqrt(2.0)) <= 1e-15
    # (c) an orthonormal pair scaled by 2 and 1/2 plus a third orthonormal
    #     vector: I - G = diag(-3, 3/4, 0), LOO = 3 (max eig 3/4)
    e3 = O.canonical_e(7, n)
    got = O.loss_of_orthogonality([O.tt_scale(e1, 2.0), O.tt_scale(e2, 0.5), e3])
    assert abs(got - 3.0) <= 1e-14
    # (d) an exactly orthonormal set of rank-2 TTs: LOO at round-off
    Q = [O.tt_scale(O.tt_add([1.0, s], [O.canonical_e(j, n), O.canonical_e(j + 20, n)]), 1 / np.sqrt(2.0))
         for j, s in ((1, 1.0), (2, -1.0), (3, 1.0))]
    assert O.loss_of_orthogonality(Q) <= 1e-15
