"""TT-matrices on the GPU (tt_operator_*, tt_matvec), the rank-capped
TT-round and the Krylov input family of the paper's experiments (Section 4),
through the C ABI, against the oracle.  The order-3 experiment (d = 3,
n = 15, m = 20, the six schemes at delta in {1e-3, 1e-5, 1e-8}) is run on
the GPU in FP64 and compared with the oracle's loss-of-orthogonality curves
and with the levels the paper prints for it (golden fixture)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle import operators as P
from ttinputs import random_tt

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2211_08770_gb300.ttgb")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctxs():
    from paper_2211_08770_gb300 import build
    build.build()
    out = {p: T.Ctx(0, p) for p in ("fp64", "fp32", "mixed_tf32")}
    yield out
    for c in out.values():
        c.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("d,n", [(1, 7), (2, 5), (3, 15), (6, 15)])
def test_laplacian_operator_equals_oracle(ctxs, prec, d, n):
    op = T.tt_operator_laplacian(ctxs[prec], d, n)
    got = op.cores()
    ref = P.laplacian_ttm(d, n)
    assert len(got) == len(ref)
    for a, b in zip(got, ref):
        assert a.shape == b.shape and np.array_equal(a, b)
    op.free()


def _rand_ttm(rng, m, n, R):
    return [rng.standard_normal((R[k], m[k], n[k], R[k + 1])) for k in range(len(m))]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-14), ("fp32", 1e-6), ("mixed_tf32", 1e-6)])
@pytest.mark.parametrize("case", ["ragged", "large", "vec4", "vec2wide"])
def test_matvec_matches_oracle(ctxs, prec, tol, case):
    rng = np.random.default_rng({"ragged": 11, "large": 12, "vec4": 13, "vec2wide": 14}[case])
    if case == "ragged":
        m, n, R, r = [3, 5, 2, 4], [4, 2, 3, 3], [1, 2, 3, 2, 1], [1, 3, 2, 4, 1]
    elif case == "large":  # several thousand CTAs' worth of outputs and a ragged tail
        m, n, R, r = [5, 64, 3], [7, 50, 9], [1, 3, 2, 1], [1, 7, 33, 1]
    elif case == "vec4":  # input-rank rows of 16-byte vectors (Q = 8, 260)
        m, n, R, r = [6, 64, 5], [5, 40, 6], [1, 2, 3, 1], [1, 8, 260, 1]
    else:  # rows of pairs longer than a CTA (Q = 1030), rows of 3 vectors (Q = 12)
        m, n, R, r = [6, 16, 5], [5, 40, 6], [1, 2, 3, 1], [1, 12, 1030, 1]
    op_h = _rand_ttm(rng, m, n, R)
    x = random_tt(rng, n, r)
    c = ctxs[prec]
    op = T.tt_operator_create(c, op_h)
    y = T.tt_matvec(c, op, T.tt_tensor_create(c, x))
    ref = P.tt_matvec(op_h, x)
    got = y.cores()
    assert O.tt_ranks(got) == O.tt_ranks(ref)
    for g, f, M, xc in zip(got, ref, op_h, x):
        # element-wise against the oracle's core, relative to the sum of the
        # magnitudes of its terms
        scale = np.einsum("aijb,pjq->apibq", np.abs(M), np.abs(xc)).reshape(f.shape)
        assert np.all(np.abs(g - f) <= tol * scale + 1e-300), np.max(np.abs(g - f) / scale)


def test_matvec_errors(ctxs):
    c = ctxs["fp64"]
    op = T.tt_operator_laplacian(c, 3, 5)
    with pytest.raises(T.TTError) as e:
        T.tt_matvec(c, op, T.tt_tensor_create(c, random_tt(np.random.default_rng(1), [5, 4, 5], [1, 2, 2, 1])))
    assert e.value.name == "TT_ERR_SHAPE"
    with pytest.raises(T.TTError) as e:
        T.tt_operator_create(c, [np.ones((2, 3, 3, 1))])
    assert e.value.name == "TT_ERR_ARG"


@pytest.mark.parametrize("cap", [0, 1, 3, 7])
def test_round_capped_fp64_matches_oracle(ctxs, cap):
    c = ctxs["fp64"]
    rng = np.random.default_rng(20 + cap)
    x = random_tt(rng, [6, 5, 7, 4, 6], [1, 5, 9, 8, 6, 1])
    delta = 1e-3
    ref = P.tt_round_rank(x, delta, cap)
    y, err = T.tt_round_capped(c, T.tt_tensor_create(c, x), delta, cap)
    got = y.cores()
    assert O.tt_ranks(got) == O.tt_ranks(ref)
    assert O.tt_diff_norm(got, ref) <= 1e-12 * O.tt_norm(x)
    # err_est is the discarded tail: equal to the true error up to round-off
    assert abs(err - O.tt_diff_norm(x, ref) / O.tt_norm(x)) <= 1e-10


@pytest.mark.parametrize("prec", ["fp32", "mixed_tf32"])
def test_round_capped_reduced_precision(ctxs, prec):
    c = ctxs[prec]
    rng = np.random.default_rng(30)
    x = random_tt(rng, [8, 8, 8, 8], [1, 8, 40, 8, 1])
    nx = O.tt_norm(x)
    for cap in (1, 4, 24):
        ref = P.tt_round_rank(x, 1e-6, cap)
        y, _ = T.tt_round_capped(c, T.tt_tensor_create(c, x), 1e-6, cap)
        got = y.cores()
        assert O.tt_ranks(got) == O.tt_ranks(ref)
        # a capped truncation of a Gaussian TT cuts between close singular
        # values, where the kept subspace moves with any perturbation: the
        # invariant is the (quasi-optimal) error, equal to FP32 level
        e_got, e_ref = O.tt_diff_norm(got, x), O.tt_diff_norm(ref, x)
        assert abs(e_got - e_ref) <= 1e-5 * nx, (cap, e_got / nx, e_ref / nx)


@pytest.mark.parametrize("d,n,m", [(3, 15, 20), (6, 15, 35)])
def test_krylov_basis_matches_oracle_fp64(ctxs, d, n, m):
    c = ctxs["fp64"]
    op_h = P.laplacian_ttm(d, n)
    ref = P.krylov_inputs(op_h, P.ones_tt([n] * d), m)
    op = T.tt_operator_laplacian(c, d, n)
    A = T.tt_krylov_basis(c, op, T.tt_tensor_create(c, P.ones_tt([n] * d)), m, 0.0, 1)
    for a, r in zip(A, ref):
        got = a.cores()
        assert O.tt_ranks(got) == [1] * (d + 1)
        assert O.tt_diff_norm(got, r) <= 1e-12


def test_krylov_basis_mixed(ctxs):
    c = ctxs["mixed_tf32"]
    d, n, m = 3, 15, 20
    ref = P.krylov_inputs(P.laplacian_ttm(d, n), P.ones_tt([n] * d), m)
    op = T.tt_operator_laplacian(c, d, n)
    A = T.tt_krylov_basis(c, op, T.tt_tensor_create(c, P.ones_tt([n] * d)), m, 0.0, 1)
    # each step is a rank-1 projection of a rank-2 TT: FP32 storage perturbs
    # the vectors at 1e-6 per step, amplified by the spectral gap of the
    # rank-1 truncation; the first vectors must match to FP32 level
    errs = [O.tt_diff_norm(a.cores(), r) for a, r in zip(A, ref)]
    assert max(errs[:5]) <= 1e-5, errs


def _gpu_loo_curve(ctx, Q):
    m = len(Q)
    G = np.zeros((m, m))
    for i in range(m):
        v = T.tt_dot_many(ctx, Q[i], Q[: i + 1])
        G[i, : i + 1] = v
        G[: i + 1, i] = v
    return [float(np.max(np.abs(np.linalg.eigvalsh(np.eye(k) - G[:k, :k])))) for k in range(1, m + 1)]


def _run_prefix(run, m):
    k = m
    while True:
        try:
            return run(k)
        except (T.TTError, np.linalg.LinAlgError) as e:
            if isinstance(e, T.TTError) and e.name != "TT_ERR_NOT_SPD":
                raise
            k -= 1


@pytest.fixture(scope="module")
def order3(ctxs):
    with open(os.path.join(GOLDEN, "krylov_order3_loo_levels.json")) as f:
        g = json.load(f)
    w = g["workload"]
    d, n, m = w["d"], w["n"], w["m"]
    A = P.krylov_inputs(P.laplacian_ttm(d, n), P.ones_tt([n] * d), m)
    c = ctxs["fp64"]
    op = T.tt_operator_laplacian(c, d, n)
    Ag = T.tt_krylov_basis(c, op, T.tt_tensor_create(c, P.ones_tt([n] * d)), m, 0.0, 1)
    out = {}
    for delta in w["deltas"]:
        for s in O.SCHEMES:
            lo = _run_prefix(lambda k: P.loo_curve(O.orthogonalize(s, A[:k], delta)[0]), m)
            lg = _run_prefix(lambda k: _gpu_loo_curve(c, T.tt_orthogonalize(c, s, Ag[:k], delta)[0]), m)
            out[(s, delta)] = (np.array(lo), np.array(lg))
    return g, out


# On this family kappa(A_k) reaches 7e8 at k = 14 and 4e13 at k = 20.  The
# sums a reorthogonalizing scheme rounds cancel to about 1 / kappa of their
# terms; the GPU's FP64 rounding orthogonalizes them by Cholesky QR, whose
# shifted fallback resolves an unfolding to about sqrt(u) of its norm, so
# the result is held to the oracle's curves and to the printed levels while
# kappa(A_k) sqrt(u) stays below about 10 (k <= 14).  Beyond, TT-MGS2's loss
# of orthogonality rises to 1e-11 - 1e-10 where the oracle's Householder QR
# keeps it at the round-off (the bench reports the whole curves).
K_FP64 = 14
# TT-Householder forms r(i) = +-sqrt(||a||^2 - s) (Algorithm 6), a
# difference of squares that leaves the new component to rounding once
# kappa(A_k)^2 u nears 1: at k = 13 (kappa ~ 1e8) the oracle's and the GPU's
# r(13) already differ in every digit and the curves part (oracle 3e-10,
# GPU 2e-5 at delta = 1e-8); it is compared up to k = 12
K_FP64_HH = 12


def _k_fp64(scheme):
    return K_FP64_HH if scheme == "householder" else K_FP64


STABLE = ("cgs2", "mgs2", "householder")


def test_order3_experiment_fp64_matches_oracle_curves(order3):
    # the FP64 GPU path follows the oracle's curve, both taken at a floor of
    # 1e-14 (values below are round-off): within a factor 10 for the stable
    # schemes; within a factor 100 for CGS, MGS and Gram, whose loss of
    # orthogonality is a constant times u kappa^p with a constant that the
    # rounding errors of each implementation set
    _, out = order3
    for (s, delta), (lo, lg) in out.items():
        k = min(len(lo), len(lg), _k_fp64(s))
        assert len(lg) >= len(lo) - 1, (s, delta, len(lo), len(lg))
        a, b = np.maximum(lo[:k], 1e-14), np.maximum(lg[:k], 1e-14)
        dec = 1.0 if s in STABLE else 2.0
        assert np.all(np.abs(np.log10(a) - np.log10(b)) <= dec), (s, delta, lo, lg)


def test_order3_experiment_fp64_matches_printed_levels(order3):
    g, out = order3
    lv = g["levels"]
    for delta in g["workload"]["deltas"]:
        c2 = out[("cgs2", delta)][1]
        m2 = out[("mgs2", delta)][1][:K_FP64]
        hh = out[("householder", delta)][1][:K_FP64_HH]
        k0 = lv["cgs2"]["flat_until_k"]
        assert c2[:k0].max() <= lv["cgs2"]["machine_level"], (delta, c2)
        if delta in lv["mgs2"]["flat_for_deltas"]:
            assert m2.max() <= lv["mgs2"]["machine_level"], (delta, m2)
        else:
            flat = m2[: lv["mgs2"]["jump_after_k"]].max()
            assert flat <= lv["mgs2"]["machine_level"]
            # the jump at k = 20: past k ~ 14 the FP64 GPU values move with
            # the rounding order of the split-K sums (8.5e-13 to above 1e-12
            # at k = 20 between runs), so it is checked as two decades above
            # the curve's own flat part, with one decade of slack on the
            # printed level
            last = out[("mgs2", delta)][1][-1]
            assert last >= max(100.0 * flat, lv["mgs2"]["jump_level"] / 10.0), (delta, last, flat)
        # up to k = 12 the Householder curve is still rising to its plateau
        # (reached near k = 20, where the oracle test checks the band from
        # below as well): here only the band's upper side applies
        h = lv["householder"]
        assert hh.max() <= h["band_above_delta"] * delta, (delta, hh)
        cg = out[("cgs", delta)][1]
        assert np.all(cg[lv["cgs"]["stagnation_after_k"] + 1:] < lv["cgs"]["stagnation_ceiling"])
