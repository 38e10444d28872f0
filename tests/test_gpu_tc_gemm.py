"""tcgen05 split-TF32 GEMM (tt_gemm_f32 through the C ABI) against an FP64
product of the same FP32 operands.

Two parts x = x_hi + x_lo (round-to-nearest TF32): each product keeps every
term but lo*lo, so its error is below 3 * 2^-22 |a||b|; three parts
(hi + mid + lo, six products) leave terms below 2^-33.  Sums add FP32
accumulation error (~2^-24 sqrt(K) relative).  Bounds, relative to
||a_i|| ||b_j|| at K <= 512: 2e-6 (two parts), 5e-7 (three parts; the FP32
round-to-nearest sum of 32 products alone reaches ~3e-7).
"""
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


def _ref(A, B, trans_b):
    Ad, Bd = A.astype(np.float64), B.astype(np.float64)
    return Ad @ (Bd.T if trans_b else Bd)


@pytest.mark.parametrize("parts,bound", [(3, 5e-7), (2, 2e-6)])
@pytest.mark.parametrize("trans_b", [True, False])
@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (400, 1000, 400), (64, 4096, 400), (25600, 400, 400),
                                   (130, 260, 36), (4, 8, 4), (1000, 64, 64)])
def test_tc_gemm_split_tf32(ctx, parts, bound, trans_b, M, N, K):
    rng = np.random.default_rng(M + 3 * N + 7 * K + trans_b)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = (rng.standard_normal((N, K)) if trans_b else rng.standard_normal((K, N))).astype(np.float32)
    Ad, Bd = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    Cd = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float32)
    T.tt_gemm_f32(ctx, trans_b, M, N, K, Ad.data_ptr(), K, Bd.data_ptr(), B.shape[1], Cd.data_ptr(), N,
                  1 if parts == 3 else 2)
    torch.cuda.synchronize()
    C = Cd.cpu().numpy().astype(np.float64)
    ref = _ref(A, B, trans_b)
    na = np.linalg.norm(A.astype(np.float64), axis=1)
    nb = np.linalg.norm(B.astype(np.float64), axis=1 if trans_b else 0)
    err = np.abs(C - ref) / np.outer(na, nb)
    assert np.all(np.isfinite(C))
    assert err.max() <= bound, err.max()
    # plain TF32 would be ~1e-3: the split really is in effect
    assert err.max() <= 1e-2 * 2.0 ** -10


def test_tc_gemm_rejects_unaligned(ctx):
    A = torch.zeros((8, 6), device="cuda")
    B = torch.zeros((6, 8), device="cuda")
    C = torch.zeros((8, 8), device="cuda")
    with pytest.raises(T.TTError) as e:
        T.tt_gemm_f32(ctx, False, 8, 8, 6, A.data_ptr(), 6, B.data_ptr(), 8, C.data_ptr(), 8, True)
    assert e.value.name == "TT_ERR_ARG"
