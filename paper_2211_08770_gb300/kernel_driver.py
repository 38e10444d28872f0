"""Runs one hot kernel of TT-round three times at a given shape, for
profiling it in isolation (e.g. under ncu):

    python -m paper_2211_08770_gb300.kernel_driver gemm   # apply Q = T X, 400 x 25600 x 400 (FP32)
    python -m paper_2211_08770_gb300.kernel_driver gram   # tensor-core Gram X X^T, n = 400, K = 25600
    python -m paper_2211_08770_gb300.kernel_driver chol   # Cholesky + inverse, n = 256 (FP32)
    python -m paper_2211_08770_gb300.kernel_driver chol400  # the blocked r = 400 factorization
    python -m paper_2211_08770_gb300.kernel_driver rgemm  # r x r product, 400 x 400 x 400 (FP32)

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
    else:
        raise SystemExit("usage: kernel_driver gemm|gram|chol|chol400|rgemm")
    torch.cuda.synchronize()
    c.close()
    print("ok", which)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "")
