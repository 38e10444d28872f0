"""Pins of the oracle's TT-matrix pieces and of the Krylov input family of
the paper's experiments (Section 4): the Laplacian TT-matrix against its
dense Kronecker sum, the TT matrix-vector product against dense brute force,
the rank-capped rounding against Eckart-Young (d = 2) and a dense TT-SVD
with a rank cap written here, the Krylov family against the same process run
on dense tensors, and the loss-of-orthogonality curves of the order-3
experiment against the levels the paper prints for it (golden fixture)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle import operators as P
from ttinputs import random_tt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense_laplacian(d, n):
    # Kronecker sum written out: sum_k I x .. x L x .. x I
    L = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    out = np.zeros((n ** d, n ** d))
    for k in range(d):
        term = np.ones((1, 1))
        for j in range(d):
            term = np.kron(term, L if j == k else np.eye(n))
        out += term
    return out


@pytest.mark.parametrize("d,n", [(1, 5), (2, 4), (3, 5), (4, 3)])
def test_laplacian_ttm_is_the_kronecker_sum(d, n):
    op = P.laplacian_ttm(d, n)
    ranks = [c.shape[0] for c in op] + [op[-1].shape[3]]
    assert ranks == ([1] + [2] * (d - 1) + [1] if d > 1 else [1, 1])
    assert np.array_equal(P.ttm_full(op), _dense_laplacian(d, n))


def _rand_ttm(rng, m, n, R):
    return [rng.standard_normal((R[k], m[k], n[k], R[k + 1])) for k in range(len(m))]


def test_matvec_dense_brute_force():
    rng = np.random.default_rng(3)
    m, n, R, r = [3, 5, 2, 4], [4, 2, 3, 3], [1, 2, 3, 2, 1], [1, 3, 2, 4, 1]
    op = _rand_ttm(rng, m, n, R)
    x = random_tt(rng, n, r)
    y = P.tt_matvec(op, x)
    assert O.tt_ranks(y) == [a * b for a, b in zip(R, r)]
    M = P.ttm_full(op)
    ref = M @ O.tt_full(x).ravel()
    # y(i) = sum_j M(i, j) x(j) with explicit loops over one output row
    i0 = 7
    row = sum(M[i0, j] * O.tt_full(x).ravel()[j] for j in range(M.shape[1]))
    assert abs(row - ref[i0]) <= 1e-12 * np.abs(M[i0]).sum() * np.abs(O.tt_full(x)).max()
    assert np.allclose(O.tt_full(y).ravel(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    with pytest.raises(ValueError):
        P.tt_matvec(op, random_tt(rng, [4, 2, 3, 4], r))


@pytest.mark.parametrize("cap", [1, 2, 5])
def test_rank_capped_round_d2_is_best_rank_approximation(cap):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((9, 7))
    x = [A.reshape(1, 9, 7), np.eye(7).reshape(7, 7, 1)]
    y = P.tt_round_rank(x, 0.0, cap)
    U, S, Vt = np.linalg.svd(A)
    best = (U[:, :cap] * S[:cap]) @ Vt[:cap]
    assert O.tt_ranks(y) == [1, cap, 1]
    assert np.allclose(O.tt_full(y), best, atol=1e-12)


def _dense_tt_svd_capped(F, cap):
    # sequential truncated SVDs of the dense tensor's unfoldings, rank <= cap
    n = F.shape
    C = F.reshape(n[0], -1)
    r = 1
    cores = []
    for k in range(len(n) - 1):
        U, S, Vt = np.linalg.svd(C.reshape(r * n[k], -1), full_matrices=False)
        rk = min(cap, len(S))
        cores.append(U[:, :rk].reshape(r, n[k], rk))
        C = S[:rk, None] * Vt[:rk]
        r = rk
    cores.append(C.reshape(r, n[-1], 1))
    return cores


@pytest.mark.parametrize("cap", [1, 3])
def test_rank_capped_round_equals_dense_tt_svd(cap):
    rng = np.random.default_rng(5)
    x = random_tt(rng, [4, 5, 3, 4], [1, 4, 6, 3, 1])
    y = P.tt_round_rank(x, 0.0, cap)
    z = _dense_tt_svd_capped(O.tt_full(x), cap)
    assert O.tt_ranks(y) == O.tt_ranks(z)
    assert np.allclose(O.tt_full(y), O.tt_full(z), atol=1e-11 * np.abs(O.tt_full(x)).max())
    # no cap: the plain rounding
    assert np.array_equal(O.tt_ranks(P.tt_round_rank(x, 1e-10, 0)), O.tt_ranks(O.tt_round(x, 1e-10)))


def test_krylov_family_equals_the_dense_process():
    d, n, m = 3, 6, 6
    op = P.laplacian_ttm(d, n)
    A = P.krylov_inputs(op, P.ones_tt([n] * d), m)
    Ld = _dense_laplacian(d, n)
    x = np.ones([n] * d)
    for j in range(m):
        a = O.tt_full(_dense_tt_svd_capped(x, 1))
        a /= np.linalg.norm(a)
        assert O.tt_ranks(A[j]) == [1] * (d + 1)
        assert np.allclose(O.tt_full(A[j]), a, atol=1e-12)
        x = (-(Ld @ a.ravel())).reshape([n] * d)
    # the first vector is the normalised ones tensor
    assert np.allclose(O.tt_full(A[0]), np.full([n] * d, n ** (-d / 2)), atol=1e-15)


def test_loo_curve_is_prefix_loo():
    rng = np.random.default_rng(6)
    Q = [random_tt(rng, [3, 4, 2], [1, 2, 2, 1]) for _ in range(4)]
    c = P.loo_curve(Q)
    for k in range(1, 5):
        assert abs(c[k - 1] - O.loss_of_orthogonality(Q[:k])) <= 1e-12 * max(1.0, c[k - 1])


def _kappas(A):
    Ad = np.column_stack([O.tt_full(a).ravel() for a in A])
    out = []
    for k in range(1, len(A) + 1):
        s = np.linalg.svd(Ad[:, :k], compute_uv=False)
        out.append(s[0] / s[-1])
    return np.array(out)


def _run(scheme, A, delta):
    # TT-Gram: the Cholesky of the Gram matrix breaks down once kappa(A_k)^2
    # passes 1/u; the curve is that of the longest prefix that factors
    # (the first k outputs of Algorithm 5 depend on the first k inputs only)
    k = len(A)
    while True:
        try:
            return P.loo_curve(O.orthogonalize(scheme, A[:k], delta)[0])
        except np.linalg.LinAlgError:
            k -= 1


@pytest.fixture(scope="module")
def order3():
    with open(os.path.join(GOLDEN, "krylov_order3_loo_levels.json")) as f:
        g = json.load(f)
    w = g["workload"]
    op = P.laplacian_ttm(w["d"], w["n"])
    A = P.krylov_inputs(op, P.ones_tt([w["n"]] * w["d"]), w["m"])
    return g, A, _kappas(A)


def test_order3_reorthogonalized_schemes_match_printed_levels(order3):
    g, A, _ = order3
    lv = g["levels"]
    for delta in g["workload"]["deltas"]:
        c2 = np.array(_run("cgs2", A, delta))
        m2 = np.array(_run("mgs2", A, delta))
        k0 = lv["cgs2"]["flat_until_k"]
        assert c2[:k0].max() <= lv["cgs2"]["machine_level"], (delta, c2)
        if delta in lv["cgs2"]["rises_for_deltas"]:
            assert c2[-1] > 100 * c2[:k0].max(), (delta, c2)
        else:
            assert c2.max() <= lv["cgs2"]["machine_level"], (delta, c2)
        if delta in lv["mgs2"]["flat_for_deltas"]:
            assert m2.max() <= lv["mgs2"]["machine_level"], (delta, m2)
        else:
            kj = lv["mgs2"]["jump_after_k"]
            assert m2[:kj].max() <= lv["mgs2"]["machine_level"], (delta, m2)
            assert m2[-1] >= lv["mgs2"]["jump_level"], (delta, m2)


def test_order3_householder_stagnates_around_delta(order3):
    g, A, _ = order3
    h = g["levels"]["householder"]
    for delta in g["workload"]["deltas"]:
        c = np.array(_run("householder", A, delta))
        assert delta / h["band_below_delta"] <= c[-1] <= h["band_above_delta"] * delta, (delta, c)


def test_order3_mgs_follows_kappa_cgs_and_gram_follow_kappa_squared(order3):
    g, A, kap = order3
    lv = g["levels"]
    delta = 1e-8
    mgs = np.array(_run("mgs", A, delta))
    cgs = np.array(_run("cgs", A, delta))
    gram = np.array(_run("gram", A, delta))
    # slopes in log-log against kappa over the range where the curves are
    # above the round-off and below O(1)
    def slope(loo, x, lo=1e-12, hi=1e-2):
        sel = (loo > lo) & (loo < hi)
        return np.polyfit(np.log10(x[sel]), np.log10(loo[sel]), 1)[0]
    a, b = lv["mgs"]["slope_vs_log_kappa"]
    assert a <= slope(mgs, kap[: len(mgs)]) <= b
    a, b = lv["gram"]["slope_vs_log_kappa2"]
    assert a <= slope(gram, kap[: len(gram)] ** 2) <= b
    assert a <= slope(cgs, kap[: len(cgs)] ** 2) <= b
    k0 = lv["cgs"]["stagnation_after_k"]
    assert np.all(cgs[k0 + 1:] < lv["cgs"]["stagnation_ceiling"]) and cgs[-1] > 1e-1
