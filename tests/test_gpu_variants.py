"""Rounding variants and the implicit-Q TT-Householder on the GPU, through
the C ABI, against the oracle: Gram-SVD rounding (FP64 agrees with the
oracle's TT-round to the method's sqrt(r u) resolution), randomized rounding
with the same random TT on both sides, and the Householder TT-vectors with
Q applied implicitly."""
import numpy as np
import pytest

import oracle as O
from oracle import variants as V
from ttinputs import coefficients, random_tt, random_tts

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2211_08770_gb300.ttgb")


@pytest.fixture(scope="module")
def ctxs():
    from paper_2211_08770_gb300 import build
    build.build()
    out = {p: T.Ctx(0, p) for p in ("fp64", "fp32", "mixed_tf32")}
    yield out
    for c in out.values():
        c.close()


def _sum(seed, m, d, n, r):
    return O.tt_add(list(coefficients(seed + 1, m)), random_tts(seed, m, d, n, r))


def _decaying(seed, n, terms, base=3.0):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(terms):
        vs = [rng.standard_normal(k) for k in n]
        out.append([(base ** -j) * vs[0].reshape(1, -1, 1)] + [v.reshape(1, -1, 1) for v in vs[1:]])
    return O.tt_add([1.0] * terms, out)


CASES = {
    "sum_d5": (lambda: _sum(1, 5, 5, 8, 4), 1e-6),
    "decaying": (lambda: _decaying(2, [6, 5, 7, 6, 5], 12), 1e-4),
    # delta well above the Gram route's sqrt(r u) resolution (~1e-7), so
    # that no singular value falls within it of the threshold
    "ragged_sum": (lambda: _sum(3, 3, 4, 11, 9), 1e-6),
    "wide_first": (lambda: _sum(4, 6, 4, 3, 5), 1e-6),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_gram_svd_fp64_matches_tt_round(ctxs, case):
    make, delta = CASES[case]
    x = make()
    c = ctxs["fp64"]
    y, err = T.tt_round_gram_svd(c, T.tt_tensor_create(c, x), delta)
    got = y.cores()
    ref = O.tt_round(x, delta)
    nx = O.tt_norm(x)
    assert O.tt_ranks(got) == O.tt_ranks(ref) == O.tt_ranks(V.tt_round_gram_svd(x, delta))
    # the same tensor as TT-round up to the Gram route's sqrt(r u) resolution
    assert O.tt_diff_norm(got, ref) <= 1e-7 * nx
    assert O.tt_diff_norm(got, x) <= (delta + 1e-7) * nx
    assert err <= delta * (1 + 1e-6)


def test_gram_svd_capped_and_redundant(ctxs):
    c = ctxs["fp64"]
    x = random_tt(np.random.default_rng(7), [5, 6, 5, 4], [1, 3, 4, 3, 1])
    z = O.tt_add([1.0, 1.0, -1.0], [x, x, x])
    y, _ = T.tt_round_gram_svd(c, T.tt_tensor_create(c, z), 1e-10)
    assert y.ranks == O.tt_ranks(x)
    assert O.tt_diff_norm(y.cores(), x) <= 1e-7 * O.tt_norm(x)
    from oracle.operators import tt_round_rank
    w = _decaying(8, [6, 7, 6], 9)
    for cap in (1, 3):
        y, _ = T.tt_round_gram_svd(c, T.tt_tensor_create(c, w), 0.0, cap)
        ref = tt_round_rank(w, 0.0, cap)
        assert y.ranks == O.tt_ranks(ref)
        assert O.tt_diff_norm(y.cores(), ref) <= 1e-7 * O.tt_norm(w)


@pytest.mark.parametrize("prec", ["fp32", "mixed_tf32"])
def test_gram_svd_reduced_precision_bound(ctxs, prec):
    # FP32 Grams resolve sqrt(r u_32) ~ 1e-3 of ||x||: checked at delta = 1e-2
    c = ctxs[prec]
    x = _decaying(9, [6, 5, 7, 6], 10, base=2.0)
    delta = 1e-2
    y, _ = T.tt_round_gram_svd(c, T.tt_tensor_create(c, x), delta)
    assert O.tt_diff_norm(y.cores(), x) <= (delta + 3e-3) * O.tt_norm(x)


def _sketch(seed, n, l):
    return random_tt(np.random.default_rng(seed), n, [1] + [l] * (len(n) - 1) + [1])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("mixed_tf32", 1e-5)])
def test_randomized_exact_recovery(ctxs, prec, tol):
    c = ctxs[prec]
    x = _sum(10, 3, 5, 6, 3)
    z = O.tt_add([1.0, 1.0, -1.0], [x, x, x])
    om = _sketch(11, [6] * 5, 12)
    y = T.tt_round_randomized(c, T.tt_tensor_create(c, z), T.tt_tensor_create(c, om))
    assert max(y.ranks) <= 12
    assert O.tt_diff_norm(y.cores(), x) <= tol * O.tt_norm(x)


@pytest.mark.parametrize("seed", range(3))
def test_randomized_fp64_matches_oracle_with_the_same_sketch(ctxs, seed):
    c = ctxs["fp64"]
    n = [7, 6, 8, 7, 5]
    x = _decaying(20 + seed, n, 14)
    om = _sketch(30 + seed, n, 9)
    y = T.tt_round_randomized(c, T.tt_tensor_create(c, x), T.tt_tensor_create(c, om))
    ref = V.tt_round_randomized(x, om)
    assert y.ranks == O.tt_ranks(ref)
    # the projection onto the sketch's range is the same tensor; its
    # numerical value depends on the sketch's conditioning
    assert O.tt_diff_norm(y.cores(), ref) <= 1e-9 * O.tt_norm(x)
    # and the same with the TT-round at delta after it
    y2 = T.tt_round_randomized(c, T.tt_tensor_create(c, x), T.tt_tensor_create(c, om), 1e-3)
    ref2 = V.tt_round_randomized(x, om, delta=1e-3)
    assert y2.ranks == O.tt_ranks(ref2)
    assert O.tt_diff_norm(y2.cores(), ref2) <= 1e-9 * O.tt_norm(x)


def test_randomized_errors(ctxs):
    c = ctxs["fp64"]
    x = T.tt_tensor_create(c, _sum(12, 2, 3, 5, 2))
    om = T.tt_tensor_create(c, _sketch(13, [5, 5, 4], 4))
    with pytest.raises(T.TTError) as e:
        T.tt_round_randomized(c, x, om)
    assert e.value.name == "TT_ERR_SHAPE"


def _hh_inputs(seed=9, m=5):
    xs = random_tts(seed, m, 4, 5, 3)
    return [O.tt_scale(x, 1.0 / O.tt_norm(x)) for x in xs]


@pytest.mark.parametrize("prec", ["fp64", "mixed_tf32"])
def test_householder_vectors_and_implicit_q(ctxs, prec):
    c = ctxs[prec]
    A = _hh_inputs()
    m = len(A)
    n = [a.shape[1] for a in A[0]]
    delta = 1e-10 if prec == "fp64" else 1e-6
    tol = 1e-11 if prec == "fp64" else 1e-5
    Ah = [T.tt_tensor_create(c, a) for a in A]
    U, R, nr = T.tt_householder_vectors(c, Ah, delta)
    Qo, Ro, no, Uo = O.tt_householder(A, delta, return_u=True)
    assert nr == 3 * m
    assert np.allclose(R, Ro, atol=tol)
    for u, uo in zip(U, Uo):
        assert O.tt_diff_norm(u.cores(), uo) <= tol
    Qg, Rg, _ = T.tt_orthogonalize(c, "householder", Ah, delta)
    for j in range(m):
        e = T.tt_canonical(c, n, j)
        hq = T.tt_householder_apply(c, U[: j + 1], e)
        q, _ = T.tt_round(c, hq, delta)
        assert O.tt_diff_norm(q.cores(), Qo[j]) <= tol
        assert O.tt_diff_norm(q.cores(), Qg[j].cores()) <= tol
    # Q^T a_i: R(:, i) on the first m canonical vectors, nothing elsewhere
    for i in range(m):
        v = O.tt_full(T.tt_householder_apply(c, U, Ah[i], transpose=True).cores()).ravel(order="F")
        assert np.allclose(v[:m], R[:, i], atol=10 * tol)
        assert np.linalg.norm(v[m:]) <= 10 * tol


def test_canonical_matches_oracle(ctxs):
    c = ctxs["fp64"]
    n = [3, 4, 2]
    for j in range(24):
        assert np.array_equal(O.tt_full(T.tt_canonical(c, n, j).cores()), O.tt_full(O.canonical_e(j + 1, n)))
    with pytest.raises(T.TTError):
        T.tt_canonical(c, n, 24)
