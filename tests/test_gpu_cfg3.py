"""Orthogonalization of the recursive, ill-conditioned family of the m = 50
workload, at reduced size (order 8, mode 32, fresh rank-10 Gaussian TTs f_k,
a_1 = f_1, a_k = c a_{k-1} + (1 - c) f_k, formed on the GPU by TT sums), for
TT-MGS2, TT-CGS2 and TT-Householder (rounding after every update) and TT-Gram
(Algorithm 5 as written), through the C ABI, against the oracle.

FP64: rounding counts equal; R within 10 delta max|R| and Q within
10 m delta in TT norm (rounding after every update, a truncation whose
threshold falls next to a singular value can keep one value more or less
than the oracle's and move the running vector by up to delta of its norm,
which later projections carry into R and Q); loss of orthogonality within
10x of the oracle's.  TT-Gram amplifies the rounding errors of its R^{-1}
by the cancellation of q_i = sum_k R^{-1}(k, i) a_k (about kappa), so only
R and the order of its loss of orthogonality are compared.

Mixed precision, where the scheme's hypothesis holds for FP32 storage
(kappa u_32 << 1 for MGS2, kappa^2 u_32 << 1 for CGS2, Householder and
Gram; Section 3.4): loss of orthogonality within max(10 LOO_oracle,
10 m u_32), R within 10 (delta + kappa u_32) max|R|."""
import numpy as np
import pytest

import oracle as O
from ttinputs import cfg_orth_recursive

pytestmark = pytest.mark.gpu

T = pytest.importorskip("paper_2211_08770_gb300.ttgb")

U32 = 2.0 ** -24
SCHEMES = ("mgs2", "cgs2", "householder", "gram")
CASES = [(0.9, 6, 1e-4), (0.9, 6, 1e-6), (0.999, 6, 1e-4), (0.999, 6, 1e-6)]


def _policy(s):
    return "paper" if s == "gram" else "every_update"


def _m(s, m):
    # TT-Gram rounds the sum of all i inputs at once (ranks add up to
    # 10 i (i + 1) / 2): five inputs keep the oracle's roundings short
    return min(m, 5) if s == "gram" else m


def _oracle_case(args):
    # one oracle orthogonalization (run in a worker process)
    c, m, delta, s = args
    F = cfg_orth_recursive(0, m=m)
    A = [F[0]]
    for k in range(1, m):
        A.append(O.tt_add([c, 1.0 - c], [A[-1], F[k]]))
    ms = _m(s, m)
    Q, R, n = O.orthogonalize(s, A[:ms], delta, _policy(s))
    G = np.array([[O.tt_dot(a, b) for b in A[:ms]] for a in A[:ms]])
    ev = np.linalg.eigvalsh(G)
    return dict(F=F[:ms], Q=Q, R=R, n=n, loo=O.loss_of_orthogonality(Q), kappa=float(np.sqrt(ev[-1] / ev[0])))


@pytest.fixture(scope="module")
def ctxs():
    from paper_2211_08770_gb300 import build
    build.build()
    out = {p: T.Ctx(0, p) for p in ("fp64", "mixed_tf32")}
    yield out
    for c in out.values():
        c.close()


@pytest.fixture(scope="module")
def oracle_runs():
    # the sixteen oracle runs are independent: a pool of spawned processes
    # (the test process already holds a CUDA context) with two BLAS threads each
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    keys = [(c, m, delta, s) for c, m, delta in CASES for s in SCHEMES]
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
    os.environ["OPENBLAS_NUM_THREADS"] = os.environ["OMP_NUM_THREADS"] = "2"
    try:
        workers = max(1, min(len(keys), (os.cpu_count() or 2) // 2))
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            out = list(ex.map(_oracle_case, keys))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return dict(zip(keys, out))


def _gpu(ctx, F, c, s, delta):
    Fg = [T.tt_tensor_create(ctx, f) for f in F]
    A = [Fg[0]]
    for k in range(1, len(F)):
        A.append(T.tt_add(ctx, [c, 1.0 - c], [A[-1], Fg[k]]))
    Q, R, n = T.tt_orthogonalize(ctx, s, A, delta, _policy(s))
    return Q, R, n, T.loss_of_orthogonality(ctx, Q)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("case", CASES, ids=lambda v: "c%g_m%d_d%g" % v)
def test_recursive_family_fp64(ctxs, oracle_runs, case, scheme):
    c, m, delta = case
    o = oracle_runs[(c, m, delta, scheme)]
    Q, R, n, loo = _gpu(ctxs["fp64"], o["F"], c, scheme, delta)
    assert n == o["n"]
    if scheme == "gram":
        # one rounding per vector, after an FP64 Cholesky of FP64 dots
        assert np.max(np.abs(R - o["R"])) <= 1e-10 * np.max(np.abs(o["R"]))
        assert loo <= 1e3 * max(o["loo"], 1e-15), (loo, o["loo"])
        return
    assert np.max(np.abs(R - o["R"])) <= 10 * delta * np.max(np.abs(o["R"]))
    for q, qo in zip(Q, o["Q"]):
        assert O.tt_diff_norm(q.cores(), qo) <= 10 * len(Q) * delta
    assert loo <= 10 * o["loo"] + 1e-15 and o["loo"] <= 10 * loo + 1e-15, (loo, o["loo"])


def _fp32_hypothesis(scheme, kappa):
    return kappa * U32 < 1e-3 if scheme == "mgs2" else kappa ** 2 * U32 < 1e-3


# c = 0.9 (kappa ~ 40): every scheme's FP32 hypothesis holds; c = 0.999
# (kappa ~ 5e3): only MGS2's (kappa^2 u_32 ~ 1 breaks CGS2, Householder's
# r(i) = sqrt(||a||^2 - s) and Gram's Cholesky)
MIXED = [(case, s) for case in CASES for s in SCHEMES if case[0] == 0.9 or s == "mgs2"]


@pytest.mark.parametrize("case,scheme", MIXED, ids=lambda v: "c%g_m%d_d%g" % v if isinstance(v, tuple) else v)
def test_recursive_family_mixed(ctxs, oracle_runs, case, scheme):
    c, m, delta = case
    o = oracle_runs[(c, m, delta, scheme)]
    assert _fp32_hypothesis(scheme, o["kappa"]), o["kappa"]
    Q, R, n, loo = _gpu(ctxs["mixed_tf32"], o["F"], c, scheme, delta)
    assert n == o["n"]
    assert loo <= max(10 * o["loo"], 10 * len(Q) * U32), (loo, o["loo"])
    tol = 10 * (delta + o["kappa"] * U32)
    assert np.max(np.abs(R - o["R"])) <= tol * np.max(np.abs(o["R"]))
