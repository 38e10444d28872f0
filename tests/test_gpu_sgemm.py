"""FP32 CUDA-core GEMM and Gram (the products TT-round keeps in FP32
arithmetic) through tt_gemm_f32(..., 0) and tt_gram_f32(..., 0), against an
FP64 product of the same FP32 operands.  Aligned products with enough
128 x 128 output tiles to fill half the SMs take the 128 x 128 kernel
(partial edge tiles along M, along N and along both, with warps beyond the
edge skipping their products), the others the 64 x 64 one (split over K
when it has few output tiles); all are covered.
FP32 accumulation over K terms: error below ~sqrt(K) u_32 |a_i||b_j| for
these random operands; the bound (1 + sqrt(K)) 1e-6 leaves a margin of ~10
while any indexing error is O(1)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
T = pytest.importorskip("paper_2211_08770_gb300.ttgb")


@pytest.fixture(scope="module")
def ctx():
    from paper_2211_08770_gb300 import build
    build.build()
    c = T.Ctx(0, "mixed_tf32")
    yield c
    c.close()


@pytest.mark.parametrize("trans_b", [False, True])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (3, 5, 7), (128, 128, 8), (129, 127, 13), (400, 25600, 400),
                                   (25600, 400, 400), (400, 1000, 4), (64, 640, 20), (1000, 36, 400),
                                   (257, 130, 1000), (1000, 10000, 64), (9000, 1000, 33), (1030, 2000, 50)])
def test_sgemm(ctx, trans_b, M, N, K):
    rng = np.random.default_rng(M + 5 * N + 11 * K + trans_b)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = (rng.standard_normal((N, K)) if trans_b else rng.standard_normal((K, N))).astype(np.float32)
    Ad, Bd = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    Cd = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float32)
    T.tt_gemm_f32(ctx, trans_b, M, N, K, Ad.data_ptr(), K, Bd.data_ptr(), B.shape[1], Cd.data_ptr(), N, 0)
    torch.cuda.synchronize()
    C = Cd.cpu().numpy().astype(np.float64)
    Ad64, Bd64 = A.astype(np.float64), B.astype(np.float64)
    ref = Ad64 @ (Bd64.T if trans_b else Bd64)
    na = np.linalg.norm(Ad64, axis=1)
    nb = np.linalg.norm(Bd64, axis=1 if trans_b else 0)
    err = np.abs(C - ref) / np.outer(na, nb)
    assert np.all(np.isfinite(C))
    assert err.max() <= (1 + np.sqrt(K)) * 1e-6, err.max()


@pytest.mark.parametrize("n,K,ld", [(1, 1, 4), (7, 9, 12), (128, 256, 256), (130, 1000, 1000), (400, 25600, 25600),
                                    (400, 25600, 25601), (64, 3, 5)])
def test_sgram_rows(ctx, n, K, ld):
    rng = np.random.default_rng(n * 7 + K)
    X = np.zeros((n, ld), dtype=np.float32)
    X[:, :K] = rng.standard_normal((n, K))
    Xd = torch.tensor(X, device="cuda")
    G = torch.full((n, n), float("nan"), device="cuda", dtype=torch.float32)
    T.tt_gram_f32(ctx, n, K, Xd.data_ptr(), ld, G.data_ptr(), 0)
    torch.cuda.synchronize()
    Gh = G.cpu().numpy().astype(np.float64)
    Xs = X[:, :K].astype(np.float64)
    ref = Xs @ Xs.T
    d = np.sqrt(np.diag(ref))
    low = np.tril(np.ones((n, n), dtype=bool))
    # lower triangle (at least) is the Gram; the kernel writes whole tiles on or below the diagonal
    err = np.abs(Gh - ref)[low] / np.outer(d, d)[low]
    assert np.all(np.isfinite(Gh[low]))
    assert err.max() <= (1 + np.sqrt(K)) * 1e-6, err.max()
