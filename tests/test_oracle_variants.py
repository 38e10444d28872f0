"""Pins of the oracle's rounding variants (randomized, Gram-SVD) and of the
implicit-Q form of TT-Householder: exact recovery of tensors of known rank,
the d = 2 cases that reduce to the randomized range finder and to
Eckart-Young, agreement with the pinned TT-round, the error bound, and the
defining property Q^T A = R of the Householder factorization."""
import numpy as np
import pytest

import oracle as O
from oracle import variants as V
from ttinputs import coefficients, random_tt, random_tts


def _sum(seed, m, d, n, r):
    xs = random_tts(seed, m, d, n, r)
    return O.tt_add(list(coefficients(seed + 1, m)), xs)


def _sketch(seed, n, l):
    d = len(n)
    return random_tt(np.random.default_rng(seed), n, [1] + [l] * (d - 1) + [1])


def test_randomized_exact_recovery_when_sketch_rank_exceeds_tt_rank():
    x = _sum(1, 3, 5, 6, 3)  # ranks <= 9
    for z in (x, O.tt_add([1.0, 1.0, -1.0], [x, x, x])):
        y = V.tt_round_randomized(z, _sketch(2, [6] * 5, 12))
        assert max(O.tt_ranks(y)) <= 12
        assert O.tt_diff_norm(y, x) <= 1e-12 * O.tt_norm(x)


def test_randomized_d2_is_the_randomized_range_finder():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((20, 6)) @ rng.standard_normal((6, 15)) + 1e-3 * rng.standard_normal((20, 15))
    x = [A.reshape(1, 20, 15), np.eye(15).reshape(15, 15, 1)]
    om = [np.ones((1, 20, 8)), rng.standard_normal((8, 15, 1))]
    y = V.tt_round_randomized(x, om)
    Z = A @ om[1][:, :, 0].T            # the sketch A Omega^T
    P = Z @ np.linalg.pinv(Z)           # orthogonal projector on range(Z)
    assert np.allclose(O.tt_full(y), P @ A, atol=1e-12)


def _decaying(seed, n, terms):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(terms):
        vs = [rng.standard_normal(k) for k in n]
        out.append([(3.0 ** -j) * vs[0].reshape(1, -1, 1)] + [v.reshape(1, -1, 1) for v in vs[1:]])
    return O.tt_add([1.0] * terms, out)


@pytest.mark.parametrize("seed", range(4))
def test_randomized_error_close_to_optimal_with_oversampling(seed):
    n = [7, 6, 8, 7]
    x = _decaying(10 + seed, n, 16)
    target, p = 6, 6
    y = V.tt_round_randomized(x, _sketch(20 + seed, n, target + p))
    from oracle.operators import tt_round_rank
    opt = O.tt_diff_norm(tt_round_rank(x, 0.0, target), x)
    assert O.tt_diff_norm(y, x) <= 10.0 * opt


def test_randomized_then_delta_rounding_meets_the_bound():
    x = _sum(4, 4, 5, 8, 4)
    y = V.tt_round_randomized(x, _sketch(5, [8] * 5, 20), delta=1e-6)
    assert O.tt_diff_norm(y, x) <= 1e-6 * O.tt_norm(x)
    assert O.tt_ranks(y) == O.tt_ranks(O.tt_round(x, 1e-6))


@pytest.mark.parametrize("delta", [1e-1, 1e-3, 1e-6])
def test_gram_svd_equals_tt_round_on_separated_spectra(delta):
    x = _decaying(30, [6, 5, 7, 6, 5], 10)
    a, b = O.tt_round(x, delta), V.tt_round_gram_svd(x, delta)
    nx = O.tt_norm(x)
    assert O.tt_ranks(a) == O.tt_ranks(b)
    assert O.tt_diff_norm(a, b) <= 1e-8 * nx
    assert O.tt_diff_norm(b, x) <= (delta + 1e-8) * nx


@pytest.mark.parametrize("cap", [1, 3])
def test_gram_svd_d2_is_eckart_young(cap):
    rng = np.random.default_rng(6)
    A = rng.standard_normal((9, 7))
    x = [A.reshape(1, 9, 7), np.eye(7).reshape(7, 7, 1)]
    y = V.tt_round_gram_svd(x, 0.0, max_rank=cap)
    U, S, Vt = np.linalg.svd(A)
    assert np.allclose(O.tt_full(y), (U[:, :cap] * S[:cap]) @ Vt[:cap], atol=1e-10)


def test_gram_svd_exact_recovery_of_redundant_sum():
    x = random_tt(np.random.default_rng(7), [5, 6, 5, 4], [1, 3, 4, 3, 1])
    z = O.tt_add([1.0, 1.0, -1.0], [x, x, x])
    y = V.tt_round_gram_svd(z, 1e-10)
    assert O.tt_ranks(y) == O.tt_ranks(x)
    assert O.tt_diff_norm(y, x) <= 1e-7 * O.tt_norm(x)


def test_gram_svd_accuracy_floor_is_sqrt_u():
    # singular values 10^0 .. 10^-12 at one bond: those below about
    # sqrt(u) of the largest are not resolved by the Gram route
    rng = np.random.default_rng(8)
    U, _ = np.linalg.qr(rng.standard_normal((30, 13)))
    W, _ = np.linalg.qr(rng.standard_normal((25, 13)))
    A = (U * np.logspace(0, -12, 13)) @ W.T
    x = [A.reshape(1, 30, 25), np.eye(25).reshape(25, 25, 1)]
    y = V.tt_round_gram_svd(x, 0.0)
    err = np.linalg.norm(O.tt_full(y) - A) / np.linalg.norm(A)
    assert 1e-12 < err <= 1e-6


def _hh_inputs(seed=9, m=5):
    xs = random_tts(seed, m, 4, 5, 3)
    return [O.tt_scale(x, 1.0 / O.tt_norm(x)) for x in xs]


def test_householder_implicit_q_equals_explicit_q():
    A = _hh_inputs()
    Q, R, _, U = O.tt_householder(A, 1e-10, return_u=True)
    n = [c.shape[1] for c in A[0]]
    for j in range(1, len(A) + 1):
        assert O.tt_diff_norm(V.householder_q(U, j, n, 1e-10), Q[j - 1]) <= 1e-12


def test_householder_implicit_qt_a_is_r():
    # Q^T a_i = H_m ... H_1 a_i has the coefficients R(:, i) on the first m
    # canonical vectors and nothing elsewhere (to the rounding accuracy)
    A = _hh_inputs()
    m = len(A)
    _, R, _, U = O.tt_householder(A, 1e-12, return_u=True)
    n = [c.shape[1] for c in A[0]]
    for i in range(m):
        v = O.tt_full(V.householder_apply(U, A[i], transpose=True)).ravel(order="F")  # i_1 fastest
        assert np.allclose(v[:m], R[:, i], atol=1e-9)
        assert np.linalg.norm(v[m:]) <= 1e-9
    # Q Q^T x = x: the reflections are involutions
    x = A[0]
    z = V.householder_apply(U, V.householder_apply(U, x, transpose=True), transpose=False)
    assert O.tt_diff_norm(z, x) <= 1e-12


def test_householder_implicit_d1_is_lapack_q():
    rng = np.random.default_rng(10)
    M = rng.standard_normal((12, 4))
    A = [[M[:, j].reshape(1, -1, 1)] for j in range(4)]
    _, _, _, U = O.tt_householder(A, 0.0, return_u=True)
    Qr, _ = np.linalg.qr(M)
    for j in range(1, 5):
        q = V.householder_q(U, j, [12], 0.0)[0].ravel()
        assert np.allclose(q, Qr[:, j - 1], atol=1e-12)
