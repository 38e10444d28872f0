"""tcgen05 column Gram G = X^T X (the Gram of a left unfolding, contraction
over the rows of X) through tt_gram_f32(..., use_tensor_cores=2), against an
FP64 Gram of the same FP32 matrix.  TF32 keeps 10 explicit mantissa bits:
bound 4e-3 sqrt(G_ii G_jj), as for the row Gram."""
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


@pytest.mark.parametrize("m,n", [(32, 1), (100, 8), (4096, 400), (25600, 400), (25600, 64), (777, 130), (777, 132),
                                 (64, 512), (3, 20)])
def test_tc_column_gram(ctx, m, n):
    g = torch.Generator(device="cpu").manual_seed(m * 31 + n)
    Xh = torch.randn(m, n, generator=g, dtype=torch.float32)
    Xh[:, : n // 3] *= 0.01  # columns of very different norms, as in the left sweep
    X = Xh.cuda()
    G = torch.full((n, n), float("nan"), device="cuda", dtype=torch.float32)
    if (4 * n) % 16:
        # a row stride that is not a multiple of 16 bytes cannot be a TMA
        # tensor map: refused before any launch
        with pytest.raises(T.TTError) as e:
            T.tt_gram_f32(ctx, n, m, X.data_ptr(), n, G.data_ptr(), 2)
        assert e.value.name == "TT_ERR_ARG"
        return
    T.tt_gram_f32(ctx, n, m, X.data_ptr(), n, G.data_ptr(), 2)
    torch.cuda.synchronize()
    Gd = G.cpu().numpy().astype(np.float64)
    Xd = Xh.numpy().astype(np.float64)
    ref = Xd.T @ Xd
    i = np.arange(n)[:, None] // 128
    j = np.arange(n)[None, :] // 128
    mask = i >= j
    dg = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.all(np.isfinite(Gd[mask]))
    assert (np.abs(Gd - ref)[mask] / dg[mask]).max() <= 4e-3
    assert np.all(Gd[~mask] == 0.0)
