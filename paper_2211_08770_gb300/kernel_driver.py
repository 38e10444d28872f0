"""Runs one hot kernel of TT-round three times at a given shape, for
profiling it in isolation (e.g. under ncu):

    python -m paper_2211_08770_gb300.kernel_driver gemm   # apply Q = T X, 400 x 25600 x 400 (FP32)
    python -m paper_2211_08770_gb300.kernel_driver gram   # tensor-core Gram X X^T, n = 400, K = 25600
    python -m paper_2211_08770_gb300.kernel_driver chol   # Cholesky + inverse, n = 256 (FP32)
    python -m paper_2211_08770_gb300.kernel_driver chol400  # the blocked r = 400 factorization
    python -m paper_2211_08770_gb300.kernel_driver rgemm  # r x r product, 400 x 400 x 400 (FP32)
    python -m paper_2211_08770_gb300.kernel_driver matvec # Laplacian TT-matrix x rank-400 TT (d = 5, n = 64)
    python -m paper_2211_08770_gb300.kernel_driver dotstack  # CGS2 passes against 48 rank-4 vectors (stacked dots)
    python -m paper_2211_08770_gb300.kernel_driver dots   # stacked multi-dot: the Gram of 64 resident rank-60 TTs
                                                          # (d = 10, n = 64) by tt_server_add_basis, mixed
    python -m paper_2211_08770_gb300.kernel_driver grams  # event times of the row and column tensor-core Grams
                                                          # at 400 x 25600 (column Gram with 3 and 5 staging stages)
    python -m paper_2211_08770_gb300.kernel_driver pipeline  # single-rounding step, sweeps pipelined vs sequential:
                                                             # ms per step and in-step device time per kernel family

The shapes are the interior bond of the single-rounding workload (20 summed
rank-20 TTs, n = 64: rank 400, unfolding length 64 x 400)."""
import sys

import numpy as np
import torch

from . import build, ttgb as T


def main(which, r=400, K=25600, n=256):
    build.build()
    c = T.Ctx(0, "mixed_tf32")
    rng = np.random.default_rng(0)
    if which == "gemm":
        A = torch.tensor(rng.standard_normal((r, r)), dtype=torch.float32, device="cuda")
        X = torch.tensor(rng.standard_normal((r, K)), dtype=torch.float32, device="cuda")
        Y = torch.empty_like(X)
        for _ in range(3):
            T.tt_gemm_f32(c, False, r, K, r, A.data_ptr(), r, X.data_ptr(), K, Y.data_ptr(), K, 0)
    elif which == "gram":
        X = torch.tensor(rng.standard_normal((r, K)), dtype=torch.float32, device="cuda")
        G = torch.empty((r, r), dtype=torch.float32, device="cuda")
        for _ in range(3):
            T.tt_gram_f32(c, r, K, X.data_ptr(), K, G.data_ptr(), 1)
    elif which == "rgemm":
        A = torch.tensor(rng.standard_normal((r, r)), dtype=torch.float32, device="cuda")
        B = torch.tensor(rng.standard_normal((r, r)), dtype=torch.float32, device="cuda")
        Cm = torch.empty_like(A)
        for _ in range(3):
            T.tt_gemm_f32(c, False, r, r, r, A.data_ptr(), r, B.data_ptr(), r, Cm.data_ptr(), r, 0)
    elif which in ("chol", "chol400"):
        n = 400 if which == "chol400" else n
        Xh = rng.standard_normal((n, 4 * n))
        G = torch.tensor(Xh @ Xh.T, dtype=torch.float32, device="cuda")
        L = torch.empty_like(G)
        Ti = torch.empty_like(G)
        for _ in range(3):
            T.tt_cholesky_inverse(c, n, G.data_ptr(), L.data_ptr(), Ti.data_ptr())
    elif which == "matvec":
        from ttinputs import random_tt
        x = random_tt(rng, [64] * 5, [1, 64, 400, 400, 64, 1], scale="unit-core")
        xt = T.tt_tensor_create(c, x)
        op = T.tt_operator_laplacian(c, 5, 64)
        for _ in range(3):
            T.tt_matvec(c, op, xt).free()
    elif which == "dotstack":
        from ttinputs import orthonormal_basis, random_tt
        Q = orthonormal_basis(rng, [64] * 10, 48, 4)
        A = [T.tt_tensor_create(c, q) for q in Q] + [
            T.tt_tensor_create(c, random_tt(rng, [64] * 10, [1] + [60] * 9 + [1], scale="unit-core"))]
        T.tt_orthogonalize(c, "cgs2", A, 1e-6)
    elif which == "pipeline":
        pipeline_families()
    elif which == "grams":
        gram_times()
    elif which == "dots":
        from ttinputs import random_tt
        Y = [T.tt_tensor_create(c, random_tt(rng, [64] * 10, [1] + [60] * 9 + [1], scale="unit-core"))
             for _ in range(64)]
        srv = T.Server(c, workers=1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        srv.add_basis(Y)
        e1.record()
        torch.cuda.synchronize()
        print("add_basis of 64 rank-60 TTs: %.3f ms" % e0.elapsed_time(e1))
        srv.close()
        for y in Y:
            y.free()
    else:
        raise SystemExit("usage: kernel_driver gemm|gram|chol|chol400|rgemm|matvec|dotstack|pipeline|grams|dots")
    torch.cuda.synchronize()
    c.close()
    print("ok", which)


def gram_times(reps=20, r=400, K=25600):
    """Microseconds per call (CUDA events, mean of reps after a warm-up) of
    the tensor-core row Gram X X^T (X r x K) and column Gram Y^T Y (Y K x r),
    the latter with 3 and 5 raw staging stages (TTGB_COLGRAM_STAGES)."""
    import json
    import os
    rng = np.random.default_rng(0)
    X = torch.tensor(rng.standard_normal((r, K)), dtype=torch.float32, device="cuda")
    Y = X.t().contiguous()
    G = torch.empty((r, r), dtype=torch.float32, device="cuda")
    out = {}
    for stages in ("3", "5"):
        os.environ["TTGB_COLGRAM_STAGES"] = stages
        c = T.Ctx(0, "mixed_tf32")
        for name, call in (("row", lambda: T.tt_gram_f32(c, r, K, X.data_ptr(), K, G.data_ptr(), 1)),
                           ("col", lambda: T.tt_gram_f32(c, r, K, Y.data_ptr(), r, G.data_ptr(), 2))):
            if name == "row" and stages == "3":
                continue
            call()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                call()
            e1.record()
            torch.cuda.synchronize()
            out["%s%s" % (name, "" if name == "row" else "_stages" + stages)] = 1e3 * e0.elapsed_time(e1) / reps
        c.close()
    os.environ.pop("TTGB_COLGRAM_STAGES", None)
    print(json.dumps(out))


def pipeline_families(steps=10):
    """ms per step of the single-rounding workload (tt_add + tt_round(1e-6),
    mixed) with the sweeps pipelined and sequential, and for each timed
    kernel family (timed alone, in its own pass) its device time per step."""
    import json
    from ttinputs import cfg_round_sum
    al, xs = cfg_round_sum(0)
    stream = torch.cuda.Stream()
    out = {}
    for pipe in (True, False):
        for fam in (None, "chol_inv", "sgemm_f32", "gram_tf32_tc"):
            c = T.Ctx(0, "mixed_tf32", stream=stream.cuda_stream)
            c.set_pipeline(pipe)
            X = [T.tt_tensor_create(c, x) for x in xs]

            def step():
                s = T.tt_add(c, al, X)
                y, _ = T.tt_round(c, s, 1e-6)
                s.free()
                y.free()

            with torch.cuda.stream(stream):
                for _ in range(3):
                    step()
            torch.cuda.synchronize()
            c.reset_profile()
            if fam:
                c.set_profiling(True, family=fam)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                for _ in range(steps):
                    step()
                e1.record(stream)
            torch.cuda.synchronize()
            prof = c.profile() if fam else {}
            c.set_profiling(False)
            out["%s/%s" % ("pipelined" if pipe else "sequential", fam or "step")] = dict(
                ms_per_step=e0.elapsed_time(e1) / steps,
                family_ms_per_step={k: v["total_ms"] / steps for k, v in prof.items()})
            for x in X:
                x.free()
            c.close()
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "")
