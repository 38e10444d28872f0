"""Pipelined sweeps of TT-round against the sequential sweeps and the oracle.

A pipelined rounding absorbs each bond's first-pass factor before the host
has seen the bond's checks and undoes the bond when they fail, so the cases
cover: every bond passing (a random sum), left-to-right bonds that truncate
(undone and redone sequentially), right-to-left first passes that are not
healthy (an exactly rank-deficient concatenation), rank-capped boundary bonds
mixed with speculative ones, and the host copies of tt_round_to_host.  The
pipelined and sequential results have the same ranks and represent the same
tensor to the storage precision; both meet the rounding bound against the
oracle's FP64 input.
"""
import numpy as np
import pytest

import oracle as O
from ttinputs import random_tt, random_tts, coefficients

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2211_08770_gb300.ttgb")

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def pairs():
    from paper_2211_08770_gb300 import build
    build.build()
    out = {}
    for p in ("fp64", "mixed_tf32", "fp32"):
        on, off = T.Ctx(0, p), T.Ctx(0, p)
        off.set_pipeline(False)
        out[p] = (on, off)
    yield out
    for on, off in out.values():
        on.close()
        off.close()


def _sum(seed, m, d, n, r):
    xs = random_tts(seed, m, d, n, r)
    return O.tt_add(list(coefficients(seed + 1, m)), xs)


def _truncating(seed, d=6, n=12):
    # a rank-3 tensor plus a small rank-5 perturbation: at delta above the
    # perturbation every interior left-to-right bond truncates
    rng = np.random.default_rng(seed)
    base = random_tt(rng, [n] * d, [1] + [3] * (d - 1) + [1])
    pert = random_tt(rng, [n] * d, [1] + [5] * (d - 1) + [1])
    nb, npt = O.tt_norm(base), O.tt_norm(pert)
    return O.tt_add([1.0, 1e-4 * nb / npt], [base, pert])


def _duplicate(seed, d=5, n=10):
    # x + x: the concatenated unfoldings have exactly dependent rows, so the
    # right-to-left first passes are not healthy (shifted path)
    x = random_tt(np.random.default_rng(seed), [n] * d, [1] + [4] * (d - 1) + [1])
    return O.tt_add([1.0, 1.0], [x, x])


CASES = {
    "sum": (lambda: _sum(3, 6, 6, 16, 4), 1e-6),
    "truncating": (lambda: _truncating(5), 1e-3),
    "duplicate": (lambda: _duplicate(7), 1e-8),
    "boundary_capped": (lambda: _sum(9, 5, 4, 3, 6), 1e-6),  # n r_d <= r_{d-1}: rank-cap bonds
}


def _tol(prec):
    return 1e-12 if prec == "fp64" else 30 * U32


@pytest.mark.parametrize("prec", ["fp64", "mixed_tf32", "fp32"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_pipelined_matches_sequential_and_oracle(pairs, prec, case):
    make, delta = CASES[case]
    x = make()
    on, off = pairs[prec]
    nx = O.tt_norm(x)
    got = {}
    for name, c in (("on", on), ("off", off)):
        c.reset_stats()
        y, _ = T.tt_round(c, T.tt_tensor_create(c, x), delta)
        got[name] = (y.cores(), c.stats())
        y.free()
    (yon, son), (yoff, soff) = got["on"], got["off"]
    assert O.tt_ranks(yon) == O.tt_ranks(yoff)
    diff = O.tt_norm(O.tt_add([1.0, -1.0], [yon, yoff]))
    assert diff <= _tol(prec) * nx, diff / nx
    # both within the rounding bound against the FP64 input
    err = O.tt_norm(O.tt_add([1.0, -1.0], [x, yon]))
    assert err <= (delta + (1e-12 if prec == "fp64" else 1e-6)) * nx, err / nx
    # the same decisions: bonds kept whole, second passes skipped, fallbacks
    for key in ("certified_bonds", "second_pass_skips", "fallback_orth", "svd_calls"):
        assert son[key] == soff[key], (key, son[key], soff[key])


@pytest.mark.parametrize("prec", ["fp64", "mixed_tf32"])
def test_pipelined_undo_paths_taken(pairs, prec):
    # the truncating case must reach the left-to-right undo (svd_calls) and
    # the duplicate case the right-to-left one (fallback_orth); in both the
    # pipelined context took its fast path elsewhere (second passes skipped)
    on, _ = pairs[prec]
    for case, key in (("truncating", "svd_calls"), ("duplicate", "fallback_orth")):
        make, delta = CASES[case]
        on.reset_stats()
        y, _ = T.tt_round(on, T.tt_tensor_create(on, make()), delta)
        y.free()
        s = on.stats()
        assert s[key] > 0, (case, s)


def test_pipelined_round_to_host(pairs):
    x = _sum(11, 6, 6, 16, 4)
    on, off = pairs["mixed_tf32"]
    outs = {}
    for name, c in (("on", on), ("off", off)):
        h = T.tt_tensor_create(c, x)
        bufs = [np.zeros(core.size, np.float32) for core in x]
        y, _, views = T.tt_round_to_host(c, h, 1e-6, bufs)
        # the host copies equal the device result
        for v, g in zip(views, y.cores()):
            np.testing.assert_array_equal(v.astype(np.float64), g)
        outs[name] = [v.astype(np.float64) for v in views]
        y.free()
    assert O.tt_ranks(outs["on"]) == O.tt_ranks(outs["off"])
    diff = O.tt_norm(O.tt_add([1.0, -1.0], [outs["on"], outs["off"]]))
    assert diff <= 30 * U32 * O.tt_norm(x)


def test_pipelined_repeated_calls_and_orthogonalization(pairs):
    # back-to-back roundings reuse the context's streams and page-locked
    # words; a Gram-Schmidt scheme rounds through the pipeline as well
    on, off = pairs["fp64"]
    x = _sum(13, 4, 5, 8, 3)
    ys = []
    for _ in range(3):
        y, _ = T.tt_round(on, T.tt_tensor_create(on, x), 1e-9)
        ys.append(y.cores())
        y.free()
    for y in ys[1:]:
        assert O.tt_norm(O.tt_add([1.0, -1.0], [y, ys[0]])) <= 1e-12 * O.tt_norm(x)
    A = [random_tt(np.random.default_rng(20 + i), [6] * 4, [1, 3, 3, 3, 1]) for i in range(4)]
    res = {}
    for name, c in (("on", on), ("off", off)):
        Q, R, _ = T.tt_orthogonalize(c, "mgs2", [T.tt_tensor_create(c, a) for a in A], 1e-10)
        res[name] = ([q.cores() for q in Q], R)
        for q in Q:
            q.free()
    np.testing.assert_allclose(res["on"][1], res["off"][1], rtol=0, atol=1e-10 * np.abs(res["off"][1]).max())
