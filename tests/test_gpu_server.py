"""Request server (tt_server_*): roundings and single Gram-Schmidt outer
iterations against resident bases, served concurrently with admission by
device footprint.  Checked: each result in the mix equals the same request
served alone; orthogonalization steps against the oracle's one-step
Algorithms 1-4; footprint admission, refusal, cancellation and wait
timeouts (all host-side, no device fault involved)."""
import numpy as np
import pytest

import oracle as O
from ttinputs import orthonormal_basis, random_tt, rank_profile

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2211_08770_gb300.ttgb")

N = [8, 6, 5, 6, 4]


@pytest.fixture(scope="module")
def ctxs():
    from paper_2211_08770_gb300 import build
    build.build()
    out = {p: T.Ctx(0, p) for p in ("fp64", "mixed_tf32")}
    yield out
    for c in out.values():
        c.close()


def _basis(seed=40, k=12, rb=3):
    return orthonormal_basis(np.random.default_rng(seed), N, k, rb)


def _requests(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        r = int(rng.integers(2, 9))
        _, ranks = rank_profile(len(N), N, r)
        x = random_tt(rng, N, ranks)
        if i % 2 == 0:
            for c in x[:-1]:
                c *= 10.0 ** (-8.0 * np.arange(c.shape[2]) / c.shape[2])
            out.append(dict(kind="round", cores=x, delta=float(rng.choice([1e-4, 1e-7]))))
        else:
            out.append(dict(kind="orth", cores=x, delta=1e-8, k=int(rng.integers(0, 13)),
                            scheme=str(rng.choice(["cgs", "mgs", "cgs2", "mgs2"]))))
    return out


def _serve(c, srv, bid, reqs, one_by_one=False):
    xs = [T.tt_tensor_create(c, q["cores"]) for q in reqs]
    res = [None] * len(reqs)

    def sub(i):
        q = reqs[i]
        if q["kind"] == "round":
            return srv.submit_round(xs[i], q["delta"])
        return srv.submit_orth(xs[i], bid, q["k"], q["scheme"], q["delta"])

    if one_by_one:
        for i, q in enumerate(reqs):
            y, cf, _ = srv.wait(sub(i), coef_cap=q.get("k", 0) + 1)
            res[i] = (y.cores(), cf)
    else:
        tickets = [sub(i) for i in range(len(reqs))]
        for i, t in enumerate(tickets):
            y, cf, _ = srv.wait(t, coef_cap=reqs[i].get("k", 0) + 1)
            res[i] = (y.cores(), cf)
    return res


def test_result_alone_equals_result_in_mix_fp64(ctxs):
    c = ctxs["fp64"]
    Q = _basis()
    reqs = _requests(41, 24)
    mix = T.Server(c, workers=6)
    bid = mix.add_basis([T.tt_tensor_create(c, q) for q in Q])
    got_mix = _serve(c, mix, bid, reqs)
    st = mix.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    mix.close()
    alone = T.Server(c, workers=1)
    bid1 = alone.add_basis([T.tt_tensor_create(c, q) for q in Q])
    got_alone = _serve(c, alone, bid1, reqs, one_by_one=True)
    alone.close()
    for q, (ym, cm), (ya, ca) in zip(reqs, got_mix, got_alone):
        nx = O.tt_norm(q["cores"])
        assert O.tt_ranks(ym) == O.tt_ranks(ya)
        scale = nx if q["kind"] == "round" else 1.0
        assert O.tt_diff_norm(ym, ya) <= 1e-12 * scale
        assert np.allclose(cm, ca, rtol=0, atol=1e-12 * nx)


@pytest.mark.parametrize("scheme", ["cgs", "mgs", "cgs2", "mgs2"])
@pytest.mark.parametrize("k", [0, 1, 7, 12])
def test_orth_step_matches_oracle_fp64(ctxs, scheme, k):
    c = ctxs["fp64"]
    Q = _basis()
    rng = np.random.default_rng(42 + k)
    a = random_tt(rng, N, [1, 4, 5, 5, 3, 1])
    srv = T.Server(c, workers=2)
    bid = srv.add_basis([T.tt_tensor_create(c, q) for q in Q])
    x = T.tt_tensor_create(c, a)
    y, cf, (ts, tb, te) = srv.wait(srv.submit_orth(x, bid, k, scheme, 1e-9), coef_cap=k + 1)
    assert ts <= tb <= te
    q_ref, col_ref, _ = O.gs_step(a, Q[:k], 1e-9, scheme)
    got = y.cores()
    assert O.tt_ranks(got) == O.tt_ranks(q_ref)
    assert O.tt_diff_norm(got, q_ref) <= 1e-12
    na = O.tt_norm(a)
    assert np.abs(np.array(cf) - col_ref).max() <= 1e-12 * na
    srv.close()


@pytest.mark.parametrize("scheme", ["cgs2", "mgs2"])
def test_orth_step_mixed_accuracy(ctxs, scheme):
    c = ctxs["mixed_tf32"]
    Q = _basis()
    a = random_tt(np.random.default_rng(43), N, [1, 4, 5, 5, 3, 1])
    delta = 1e-6
    srv = T.Server(c, workers=2)
    bid = srv.add_basis([T.tt_tensor_create(c, q) for q in Q])
    y, cf, _ = srv.wait(srv.submit_orth(T.tt_tensor_create(c, a), bid, 12, scheme, delta), coef_cap=13)
    q_ref, col_ref, _ = O.gs_step(a, Q, delta, scheme)
    na = O.tt_norm(a)
    assert np.abs(np.array(cf) - col_ref).max() <= (delta + 1e-6) * na
    got = y.cores()
    assert O.tt_diff_norm(got, q_ref) <= 10 * (delta + 1e-6) * na / col_ref[-1]
    loo_g = O.loss_of_orthogonality(Q + [got])
    loo_o = O.loss_of_orthogonality(Q + [q_ref])
    assert loo_g <= 10 * max(loo_o, 1e-6)
    srv.close()


def test_footprint_admission_refusal_cancel_timeout(ctxs):
    c = ctxs["fp64"]
    reqs = [q for q in _requests(44, 16) if q["kind"] == "round"]
    xs = [T.tt_tensor_create(c, q["cores"]) for q in reqs]
    # the largest bound: one worker serves the requests one at a time
    probe = T.Server(c, workers=1, footprint_budget=1 << 40)
    for x in xs:
        probe.wait(probe.submit_round(x, 1e-6))[0].free()
    one = probe.stats()["footprint_peak"]
    probe.close()
    assert one > 0
    srv = T.Server(c, workers=4, footprint_budget=2 * one)
    # a request larger than the whole budget is refused at submit
    big = random_tt(np.random.default_rng(45), [16] * 6, [1, 16, 60, 60, 60, 16, 1])
    with pytest.raises(T.TTError) as e:
        srv.submit_round(T.tt_tensor_create(c, big), 1e-6)
    assert e.value.name == "TT_ERR_OOM"
    tickets = [srv.submit_round(x, 1e-6) for x in xs]
    last = tickets[-1]
    cancelled = True
    try:
        srv.cancel(last)
    except T.TTError as e:  # it may already have started
        assert e.value.name == "TT_ERR_ARG"
        cancelled = False
    with pytest.raises(T.TTError) as e:
        srv.wait(123456789)
    assert e.value.name == "TT_ERR_ARG"
    for t in tickets[:-1]:
        y, _, _ = srv.wait(t)
        y.free()
    if cancelled:
        with pytest.raises(T.TTError) as e:
            srv.wait(last)
        assert e.value.name == "TT_ERR_CANCELLED"
    else:
        srv.wait(last)[0].free()
    st = srv.stats()
    assert st["footprint_peak"] <= 2 * one
    assert st["refused"] == 1 and st["queued"] == 0 and st["running"] == 0
    assert st["completed"] == len(xs) - (1 if cancelled else 0)
    # a wait with a zero timeout on a queued request times out, the ticket stays valid
    slow = T.Server(c, workers=1)
    ts = [slow.submit_round(x, 1e-6) for x in xs]
    with pytest.raises(T.TTError) as e:
        slow.wait(ts[-1], timeout_ms=0)
    assert e.value.name == "TT_ERR_TIMEOUT"
    for t in ts:
        slow.wait(t)[0].free()
    slow.close()
    srv.close()


def test_poisson_load_small(ctxs):
    from paper_2211_08770_gb300.serve import poisson_load
    c = ctxs["mixed_tf32"]
    Q = _basis()
    srv = T.Server(c, workers=4)
    bid = srv.add_basis([T.tt_tensor_create(c, q) for q in Q])
    reqs = _requests(46, 40)
    for q in reqs:
        q["d"], q["n"] = len(N), N[0]
    out = poisson_load(srv, c, reqs, rate=200.0, basis_ids={(len(N), N[0]): bid}, seed=1)
    assert out["completed"] == len(reqs) and not out["errors"]
    assert 0 < out["p50_ms"] <= out["p99_ms"]
    srv.close()


def test_result_alone_equals_result_in_mix_mixed(ctxs):
    # the mixed path in the mix and alone: each result within the mixed
    # tolerance of the input (delta + 1e-6, relative), so two runs of one
    # request differ by at most twice that; ranks within one (a split-K sum
    # may round differently next to the threshold)
    c = ctxs["mixed_tf32"]
    Q = _basis()
    reqs = _requests(47, 16)
    mix = T.Server(c, workers=6)
    bid = mix.add_basis([T.tt_tensor_create(c, q) for q in Q])
    got_mix = _serve(c, mix, bid, reqs)
    assert mix.stats()["completed"] == len(reqs)
    mix.close()
    alone = T.Server(c, workers=1)
    bid1 = alone.add_basis([T.tt_tensor_create(c, q) for q in Q])
    got_alone = _serve(c, alone, bid1, reqs, one_by_one=True)
    alone.close()
    for q, (ym, cm), (ya, ca) in zip(reqs, got_mix, got_alone):
        tol = q["delta"] + 1e-6
        nx = O.tt_norm(q["cores"])
        assert all(abs(a - b) <= 1 for a, b in zip(O.tt_ranks(ym), O.tt_ranks(ya)))
        if q["kind"] == "round":
            assert O.tt_diff_norm(ym, q["cores"]) <= tol * nx
            assert O.tt_diff_norm(ya, q["cores"]) <= tol * nx
            assert O.tt_diff_norm(ym, ya) <= 2 * tol * nx
        else:
            assert np.abs(np.array(cm) - np.array(ca)).max() <= 2 * tol * nx
            assert O.tt_diff_norm(ym, ya) <= 20 * tol * nx / ca[-1]


def test_add_basis_while_steps_run(ctxs):
    # tt_server_add_basis grows the list of bases while workers run
    # orthogonalization steps against basis 0: each step reads the basis
    # vectors it was admitted with, and every result equals the same step
    # served alone
    import threading
    c = ctxs["fp64"]
    Q = _basis()
    srv = T.Server(c, workers=6)
    qs = [T.tt_tensor_create(c, q) for q in Q]
    bid = srv.add_basis(qs)
    rng = np.random.default_rng(48)
    xs = [random_tt(rng, N, [1, 3, 4, 4, 3, 1]) for _ in range(24)]
    hx = [T.tt_tensor_create(c, x) for x in xs]
    added = []
    stop = threading.Event()

    def grow():
        while not stop.is_set() and len(added) < 64:
            added.append(srv.add_basis(qs))

    th = threading.Thread(target=grow)
    th.start()
    try:
        tickets = [srv.submit_orth(h, bid, 12, "cgs2" if i % 2 else "mgs2", 1e-9) for i, h in enumerate(hx)]
        res = [srv.wait(t, coef_cap=13) for t in tickets]
    finally:
        stop.set()
        th.join()
    assert len(added) > 0 and len(set(added)) == len(added)
    for i, (y, cf, _) in enumerate(res):
        q_ref, col_ref, _ = O.gs_step(xs[i], Q, 1e-9, "cgs2" if i % 2 else "mgs2")
        got = y.cores()
        assert O.tt_diff_norm(got, q_ref) <= 1e-12
        assert np.abs(np.array(cf) - col_ref).max() <= 1e-12 * O.tt_norm(xs[i])
    srv.close()
