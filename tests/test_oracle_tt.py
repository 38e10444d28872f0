"""Pins of the oracle's TT primitives against what the paper and plain
linear algebra fix: dense brute force, closed forms, Eckart-Young, a dense
TT-SVD written here independently, exact recovery of known ranks and the
rounding error bound ||x - round(x)|| <= delta ||x|| (Section 2)."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from ttinputs import random_tt, rank_profile

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(seed, n, ranks):
    return random_tt(np.random.default_rng(seed), n, ranks)


def test_full_rank1_is_outer_product():
    rng = np.random.default_rng(1)
    vs = [rng.standard_normal(k) for k in (3, 4, 5)]
    cores = [v.reshape(1, -1, 1) for v in vs]
    ref = np.einsum("i,j,k->ijk", *vs)
    assert np.allclose(O.tt_full(cores), ref, rtol=0, atol=1e-14)


def test_full_matches_slice_products():
    n, ranks = [3, 4, 2, 3], [1, 2, 3, 2, 1]
    x = _rand(2, n, ranks)
    F = O.tt_full(x)
    for idx in itertools.product(*[range(k) for k in n]):
        # x(i1..id) = X_1(i1) ... X_d(id) written out with explicit loops
        v = np.ones((1, 1))
        for c, i in zip(x, idx):
            w = np.zeros((v.shape[0], c.shape[2]))
            for a in range(v.shape[0]):
                for b in range(c.shape[2]):
                    w[a, b] = sum(v[a, t] * c[t, i, b] for t in range(c.shape[0]))
            v = w
        assert abs(F[idx] - v[0, 0]) < 1e-12


def test_add_is_dense_sum_and_ranks_add():
    n, r1, r2 = [3, 4, 3, 2], [1, 2, 3, 2, 1], [1, 3, 2, 2, 1]
    x, y, z = _rand(3, n, r1), _rand(4, n, r2), _rand(5, n, r1)
    al = [0.3, -1.7, 2.5]
    s = O.tt_add(al, [x, y, z])
    ref = al[0] * O.tt_full(x) + al[1] * O.tt_full(y) + al[2] * O.tt_full(z)
    assert np.allclose(O.tt_full(s), ref, rtol=0, atol=1e-12)
    assert O.tt_ranks(s) == [1] + [a + b + c for a, b, c in zip(r1[1:-1], r2[1:-1], r1[1:-1])] + [1]


def test_add_d1_and_mode_mismatch():
    a = [np.arange(5.0).reshape(1, 5, 1)]
    b = [np.ones((1, 5, 1))]
    s = O.tt_add([2.0, -1.0], [a, b])
    assert np.allclose(s[0].ravel(), 2 * np.arange(5.0) - 1)
    with pytest.raises(ValueError):
        O.tt_add([1.0, 1.0], [a, [np.ones((1, 4, 1))]])


def test_dot_dense_and_rank1_closed_form():
    n = [4, 3, 5, 2]
    x, y = _rand(6, n, [1, 2, 4, 2, 1]), _rand(7, n, [1, 3, 2, 2, 1])
    assert abs(O.tt_dot(x, y) - float(np.sum(O.tt_full(x) * O.tt_full(y)))) < 1e-11
    rng = np.random.default_rng(8)
    u = [rng.standard_normal(k) for k in n]
    v = [rng.standard_normal(k) for k in n]
    closed = math.prod(float(a @ b) for a, b in zip(u, v))
    got = O.tt_dot([a.reshape(1, -1, 1) for a in u], [b.reshape(1, -1, 1) for b in v])
    assert abs(got - closed) < 1e-12 * max(1.0, abs(closed))


def test_canonical_basis_orthonormal_and_i1_fastest():
    n = [3, 2, 4]
    N = 24
    for j in range(1, N + 1):
        e = O.canonical_e(j, n)
        assert O.tt_ranks(e) == [1, 1, 1, 1]
        flat = O.tt_full(e).flatten(order="F")  # i_1 fastest
        assert flat[j - 1] == 1.0 and flat.sum() == 1.0
    for i in range(1, 7):
        for j in range(1, 7):
            assert O.tt_dot(O.canonical_e(i, n), O.canonical_e(j, n)) == float(i == j)
    with pytest.raises(ValueError):
        O.canonical_phi(N + 1, n)


def test_norm_and_rl_orthogonalization():
    n, ranks = [4, 5, 3, 4], [1, 3, 4, 3, 1]
    x = _rand(9, n, ranks)
    y, nrm = O.tt_orthogonalize_rl(x)
    assert abs(nrm - np.linalg.norm(O.tt_full(x))) < 1e-12 * nrm
    assert np.allclose(O.tt_full(y), O.tt_full(x), atol=1e-12 * nrm)
    for c in y[1:]:
        M = c.reshape(c.shape[0], -1)
        assert np.allclose(M @ M.T, np.eye(M.shape[0]), atol=1e-13)


def _tail_rank(S, eps):
    # independent restatement of "minimal r with the discarded tail <= eps"
    r = len(S)
    while r > 1 and math.sqrt(sum(s * s for s in S[r - 1:])) <= eps:
        r -= 1
    return r


@pytest.mark.parametrize("delta", [1e-1, 3e-2, 1e-3])
def test_round_d2_is_truncated_svd(delta):
    rng = np.random.default_rng(10)
    U, _ = np.linalg.qr(rng.standard_normal((12, 9)))
    V, _ = np.linalg.qr(rng.standard_normal((10, 9)))
    S = 2.0 ** -np.arange(9)
    A = (U * S) @ V.T
    # as a d = 2 TT: core_1 = A (1 x 12 x 10), core_2 = I (10 x 10 x 1)
    x = [A.reshape(1, 12, 10), np.eye(10).reshape(10, 10, 1)]
    y = O.tt_round(x, delta)
    Uf, Sf, Vf = np.linalg.svd(A)
    r = _tail_rank(Sf, delta * np.linalg.norm(A))
    ref = (Uf[:, :r] * Sf[:r]) @ Vf[:r]
    assert O.tt_ranks(y)[1] == r
    assert np.allclose(O.tt_full(y), ref, atol=1e-13)


def _dense_tt_svd(A, delta):
    """Dense TT-SVD [Oseledets 2011], written here independently of the
    oracle: successive truncated SVDs of the unfoldings of the dense tensor,
    per-bond threshold delta ||A|| / sqrt(d - 1)."""
    n = A.shape
    d = len(n)
    eps = delta * np.linalg.norm(A) / math.sqrt(d - 1)
    cores = []
    r_prev = 1
    C = A.copy()
    for k in range(d - 1):
        C = C.reshape(r_prev * n[k], -1)
        U, S, Vt = np.linalg.svd(C, full_matrices=False)
        r = _tail_rank(S, eps)
        cores.append(U[:, :r].reshape(r_prev, n[k], r))
        C = S[:r, None] * Vt[:r]
        r_prev = r
    cores.append(C.reshape(r_prev, n[-1], 1))
    return cores


@pytest.mark.parametrize("delta", [0.3, 0.05, 1e-3])
def test_round_equals_dense_tt_svd(delta):
    # a tensor with a decaying spectrum: sum of rank-1 terms with weights 2^-j
    rng = np.random.default_rng(11)
    n = [5, 4, 6, 3]
    terms = []
    for j in range(8):
        vs = [rng.standard_normal(k) for k in n]
        terms.append([(2.0 ** -j) * vs[0].reshape(1, -1, 1)] + [v.reshape(1, -1, 1) for v in vs[1:]])
    x = O.tt_add([1.0] * len(terms), terms)
    y = O.tt_round(x, delta)
    z = _dense_tt_svd(O.tt_full(x), delta)
    assert O.tt_ranks(y) == O.tt_ranks(z)
    assert np.allclose(O.tt_full(y), O.tt_full(z), atol=1e-11 * np.linalg.norm(O.tt_full(x)))


@pytest.mark.parametrize("seed", range(6))
def test_round_error_bound_property(seed):
    rng = np.random.default_rng(100 + seed)
    d = int(rng.integers(2, 6))
    n = [int(v) for v in rng.integers(2, 6, size=d)]
    _, ranks = rank_profile(d, n, int(rng.integers(1, 7)))
    x = random_tt(rng, n, ranks)
    delta = float(10.0 ** rng.uniform(-6, -0.3))
    y = O.tt_round(x, delta)
    F = O.tt_full(x)
    err = np.linalg.norm(F - O.tt_full(y))
    assert err <= delta * np.linalg.norm(F) * (1 + 1e-10) + 1e-13
    assert all(a <= b for a, b in zip(O.tt_ranks(y), O.tt_ranks(x)))


def test_exact_recovery_of_redundant_sum():
    n, ranks = [6, 5, 6, 5, 4], [1, 3, 4, 4, 3, 1]
    x = _rand(12, n, ranks)
    s = O.tt_add([1.0, 1.0, -1.0], [x, x, x])
    y = O.tt_round(s, 1e-12)
    assert O.tt_ranks(y) == ranks
    assert O.tt_diff_norm(x, y) <= 1e-12 * O.tt_norm(x)


def test_exact_recovery_of_gauge_padded_ranks():
    rng = np.random.default_rng(13)
    n, ranks = [5, 6, 5, 6], [1, 2, 3, 2, 1]
    x = random_tt(rng, n, ranks)
    pad = 3
    A = [np.ones((1, 1))]
    Ap = [np.ones((1, 1))]
    for k in range(1, len(n)):
        M = rng.standard_normal((ranks[k], ranks[k] + pad))
        A.append(M)
        Ap.append(np.linalg.pinv(M))  # right inverse: M @ pinv(M) = I
    A.append(np.ones((1, 1)))
    Ap.append(np.ones((1, 1)))
    y = [np.einsum("pa,aib,bq->piq", Ap[k], x[k], A[k + 1]) for k in range(len(n))]
    assert O.tt_ranks(y) == [1] + [r + pad for r in ranks[1:-1]] + [1]
    z = O.tt_round(y, 1e-12)
    assert O.tt_ranks(z) == ranks
    assert np.allclose(O.tt_full(z), O.tt_full(x), atol=1e-11 * O.tt_norm(x))


def test_round_idempotent_d1_identity_and_delta0():
    n, ranks = [4, 4, 4, 4], [1, 3, 5, 3, 1]
    x = _rand(14, n, ranks)
    y = O.tt_round(x, 0.2)
    z = O.tt_round(y, 0.2)
    assert O.tt_ranks(z) == O.tt_ranks(y)
    x1 = [np.arange(1.0, 6.0).reshape(1, 5, 1)]
    assert np.array_equal(O.tt_round(x1, 0.5)[0], x1[0])
    assert O.tt_ranks(O.tt_round(x, 0.0)) == ranks
    with pytest.raises(ValueError):
        O.tt_round(x, -1.0)


def test_diff_norm_and_bond_singular_values_dense():
    n = [4, 3, 5, 3]
    x, y = _rand(15, n, [1, 3, 4, 3, 1]), _rand(16, n, [1, 2, 3, 2, 1])
    ref = np.linalg.norm(O.tt_full(x) - O.tt_full(y))
    assert abs(O.tt_diff_norm(x, y) - ref) < 1e-12 * ref
    F = O.tt_full(x)
    sv = O.bond_singular_values(x)
    for k in range(len(n) - 1):
        Sd = np.linalg.svd(F.reshape(int(np.prod(n[: k + 1])), -1), compute_uv=False)
        m = len(sv[k])
        assert np.allclose(sv[k], Sd[:m], atol=1e-12 * Sd[0])
        assert np.all(Sd[m:] < 1e-12 * Sd[0])


def test_compression_ratio_and_gain_closed_form():
    x = _rand(17, [3, 4, 5], [1, 2, 3, 1])
    assert O.compression_ratio(x) == (1 * 3 * 2 + 2 * 4 * 3 + 3 * 5 * 1) / 60.0
    y = _rand(18, [3, 4, 5], [1, 1, 1, 1])
    assert O.compression_gain(x, y) == (6 + 24 + 15) / (3 + 4 + 5)


def test_golden_cost_table_is_well_formed():
    with open(os.path.join(GOLDEN, "tab_orth_rounding_counts.json")) as f:
        g = json.load(f)
    assert set(g["rounds_per_m"]) == {"gram", "cgs", "mgs", "cgs2", "mgs2", "householder"}
