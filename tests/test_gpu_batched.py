"""Batched TT-rounding (tt_round_batched: independent roundings of uneven
order, mode size and rank run concurrently on lanes) against the oracle and
against one tt_round per tensor.  FP64: ranks equal and 1e-12 relative
difference; mixed: the rounding bound (delta + 1e-6) ||x|| and ranks within
one of the oracle's."""
import numpy as np
import pytest

import oracle as O
from ttinputs import random_tt, rank_profile

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2211_08770_gb300.ttgb")


@pytest.fixture(scope="module")
def ctxs():
    from paper_2211_08770_gb300 import build
    build.build()
    out = {p: T.Ctx(0, p) for p in ("fp64", "mixed_tf32")}
    yield out
    for c in out.values():
        c.close()


def _mix(seed, count):
    """Uneven instances: plain random TTs, redundant sums x + y - y (exact
    rank recovery), decaying sums (bonds truncated at delta) and d = 1."""
    rng = np.random.default_rng(seed)
    xs, deltas = [], []
    for i in range(count):
        d = int(rng.integers(2, 7))
        n = int(rng.choice([4, 8, 16, 32]))
        r = int(rng.integers(2, 24))
        nn, ranks = rank_profile(d, n, r)
        kind = i % 4
        if kind == 0:
            x = random_tt(rng, nn, ranks, scale="unit-core")
        elif kind == 1:
            a = random_tt(rng, nn, ranks, scale="unit-core")
            b = random_tt(rng, nn, ranks, scale="unit-core")
            x = O.tt_add([1.0, 1.0, -1.0], [a, b, b])
        elif kind == 2:
            terms = [random_tt(rng, nn, [1] * (d + 1)) for _ in range(6)]
            x = O.tt_add([2.0 ** -(3 * j) for j in range(6)], terms)
        else:
            x = random_tt(rng, [int(rng.integers(3, 40))], [1, 1]) if i % 8 == 3 else \
                random_tt(rng, nn, ranks)
        xs.append(x)
        deltas.append(float(rng.choice([1e-3, 1e-6, 1e-9])))
    return xs, deltas


def _up(ctx, xs):
    return [T.tt_tensor_create(ctx, x) for x in xs]


@pytest.mark.parametrize("lanes", [1, 4, 8])
def test_batched_fp64_matches_oracle_and_single(ctxs, lanes):
    c = ctxs["fp64"]
    c.concurrency = lanes
    xs, deltas = _mix(100 + lanes, 24)
    hs = _up(c, xs)
    c.reset_stats()
    ys = T.tt_round_batched(c, hs, deltas)
    assert c.stats()["roundings"] >= sum(1 for x in xs if len(x) > 1)
    for x, h, dl, y in zip(xs, hs, deltas, ys):
        got = y.cores()
        ref = O.tt_round(x, dl)
        nx = O.tt_norm(x)
        assert O.tt_ranks(got) == O.tt_ranks(ref)
        assert O.tt_diff_norm(got, ref) <= 1e-12 * nx
        single, _ = T.tt_round(c, h, dl)
        assert single.ranks == y.ranks
        assert O.tt_diff_norm(got, single.cores()) <= 1e-12 * nx
    c.concurrency = 8


def test_batched_mixed_error_bound(ctxs):
    c = ctxs["mixed_tf32"]
    c.concurrency = 8
    xs, deltas = _mix(7, 32)
    deltas = [max(v, 1e-6) for v in deltas]
    ys = T.tt_round_batched(c, _up(c, xs), deltas)
    for x, dl, y in zip(xs, deltas, ys):
        got = y.cores()
        nx = O.tt_norm(x)
        assert O.tt_diff_norm(got, x) <= (dl + 1e-6) * nx
        rg, rr = O.tt_ranks(got), O.tt_ranks(O.tt_round(x, dl))
        assert all(abs(a - b) <= 1 for a, b in zip(rg, rr)), (rg, rr)


def test_batched_edge_cases(ctxs):
    c = ctxs["fp64"]
    assert T.tt_round_batched(c, [], []) == []
    xs, deltas = _mix(3, 4)
    hs = _up(c, xs)
    with pytest.raises(T.TTError) as e:
        T.tt_round_batched(c, hs, deltas[:3] + [-1.0])
    assert e.value.name == "TT_ERR_ARG"
    with pytest.raises(T.TTError) as e:
        c.concurrency = 0
    assert e.value.name == "TT_ERR_ARG"
    # one instance, more lanes than instances
    c.concurrency = 16
    (y,) = T.tt_round_batched(c, hs[:1], deltas[:1])
    assert y.ranks == O.tt_ranks(O.tt_round(xs[0], deltas[0]))
    c.concurrency = 8


def test_batched_budget_shared_by_lanes(ctxs):
    # every lane draws on the context's budget: a batch whose workspaces do
    # not fit fails with TT_ERR_OOM, returns nothing and leaves the context
    # usable with its byte count restored
    rng = np.random.default_rng(5)
    nn, ranks = rank_profile(6, 32, 40)
    xs = [random_tt(rng, nn, ranks) for _ in range(16)]
    in_bytes = sum(8 * sum(a.size for a in x) for x in xs)
    small = T.Ctx(0, "fp64", hbm_budget=int(in_bytes * 1.3) + (1 << 20))
    small.concurrency = 8
    hs = _up(small, xs)
    before = small.stats()["bytes_in_use"]
    with pytest.raises(T.TTError) as e:
        T.tt_round_batched(small, hs, [1e-8] * len(hs))
    assert e.value.name == "TT_ERR_OOM"
    assert small.stats()["bytes_in_use"] == before
    small.concurrency = 1
    y, _ = T.tt_round(small, hs[0], 1e-8)
    assert y.ranks == O.tt_ranks(O.tt_round(xs[0], 1e-8))
    y.free()
    for h in hs:
        h.free()
    small.close()
