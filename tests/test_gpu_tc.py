"""tcgen05 TF32 Gram kernel (tt_gram_f32 through the C ABI) against an FP64
Gram of the same FP32 matrix, and against the CUDA-core FP32 kernel.

TF32 keeps 10 explicit mantissa bits, so each product carries a relative
error below 2^-9; the bound used here, 4e-3 sqrt(G_ii G_jj), is that
worst-case product error summed coherently (|<x_i, x_j>| <= ||x_i|| ||x_j||).
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


def _lower_tiles_mask(n, tile):
    i = np.arange(n)[:, None] // tile
    j = np.arange(n)[None, :] // tile
    return i >= j


@pytest.mark.parametrize("n,K", [(1, 32), (7, 64), (128, 256), (130, 1000), (200, 4096), (400, 25600), (513, 96)])
def test_tc_gram_matches_fp64(ctx, n, K):
    g = torch.Generator(device="cpu").manual_seed(n * 7919 + K)
    Xh = torch.randn(n, K, generator=g, dtype=torch.float32)
    X = Xh.cuda()
    G = torch.full((n, n), float("nan"), device="cuda", dtype=torch.float32)
    T.tt_gram_f32(ctx, n, K, X.data_ptr(), K, G.data_ptr(), True)
    torch.cuda.synchronize()
    Gd = G.cpu().numpy().astype(np.float64)
    Xd = Xh.numpy().astype(np.float64)
    ref = Xd @ Xd.T
    mask = _lower_tiles_mask(n, 128)
    dg = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    err = np.abs(Gd - ref)[mask] / dg[mask]
    assert np.all(np.isfinite(Gd[mask]))
    assert err.max() <= 4e-3, err.max()
    # strictly-upper tiles are left at zero
    assert np.all(Gd[~mask] == 0.0)
    # the CUDA-core FP32 kernel on the same input
    G2 = torch.zeros((n, n), device="cuda", dtype=torch.float32)
    T.tt_gram_f32(ctx, n, K, X.data_ptr(), K, G2.data_ptr(), False)
    torch.cuda.synchronize()
    m64 = _lower_tiles_mask(n, 64)
    e2 = (np.abs(G2.cpu().numpy().astype(np.float64) - ref)[m64] / dg[m64]).max()
    assert e2 <= 1e-5


def test_tc_gram_strided_rows(ctx):
    n, K, ld = 96, 640, 1024
    Xh = torch.randn(n, ld, dtype=torch.float32)
    X = Xh.cuda()
    G = torch.zeros((n, n), device="cuda", dtype=torch.float32)
    T.tt_gram_f32(ctx, n, K, X.data_ptr(), ld, G.data_ptr(), True)
    torch.cuda.synchronize()
    Xd = Xh[:, :K].numpy().astype(np.float64)
    ref = Xd @ Xd.T
    dg = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    low = np.tril(np.ones((n, n), dtype=bool))
    assert (np.abs(G.cpu().numpy() - ref)[low] / dg[low]).max() <= 4e-3


def test_tc_gram_rejects_unaligned_stride(ctx):
    n, K = 8, 30  # 30 * 4 bytes is not a multiple of 16
    X = torch.randn(n, K, device="cuda", dtype=torch.float32)
    G = torch.zeros((n, n), device="cuda", dtype=torch.float32)
    with pytest.raises(T.TTError) as e:
        T.tt_gram_f32(ctx, n, K, X.data_ptr(), K, G.data_ptr(), True)
    assert e.value.name == "TT_ERR_ARG"


def _spd(n, seed, kappa=1e2, dtype=np.float64):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.logspace(0, -np.log10(kappa), n)
    return ((Q * ev) @ Q.T).astype(dtype)


@pytest.mark.parametrize("prec", ["fp64", "mixed_tf32"])
@pytest.mark.parametrize("n,nb", [(1, 0), (5, 0), (31, 0), (32, 0), (33, 0), (100, 0), (160, 0), (161, 0), (255, 0),
                                  (256, 0), (257, 0), (400, 0), (600, 0), (100, 32), (257, 64), (400, 128),
                                  (400, 96)])
def test_cholesky_inverse_blocked(prec, n, nb, monkeypatch):
    # nb = 0: the block size the library picks (one CTA up to 256 / 160,
    # autotuned blocks above); nb > 0 forces blocks of that size
    from paper_2211_08770_gb300 import build
    build.build()
    monkeypatch.setenv("TTGB_CHOL_NB", str(nb))
    c = T.Ctx(0, prec)
    tdt = torch.float64 if prec == "fp64" else torch.float32
    G = _spd(n, n, 1e2)
    Gd = torch.tensor(G, dtype=tdt, device="cuda")
    L = torch.empty_like(Gd)
    Ti = torch.empty_like(Gd)
    nd = T.tt_cholesky_inverse(c, n, Gd.data_ptr(), L.data_ptr(), Ti.data_ptr())
    assert nd == 0
    Lh = L.cpu().numpy().astype(np.float64)
    Th = Ti.cpu().numpy().astype(np.float64)
    tol = 1e-13 if prec == "fp64" else 2e-5
    assert np.allclose(np.triu(Lh, 1), 0) and np.allclose(np.triu(Th, 1), 0)
    assert np.linalg.norm(Lh @ Lh.T - G) <= tol * np.linalg.norm(G) * np.sqrt(n)
    assert np.linalg.norm(Th @ Lh - np.eye(n)) <= tol * 100 * np.sqrt(n)
    c.close()


@pytest.mark.parametrize("n,nb,dep", [(70, 0, (40, 65)), (70, 32, (40, 65)), (300, 64, (40, 65, 150, 299))])
def test_cholesky_inverse_drops_dependent_rows(n, nb, dep, monkeypatch):
    from paper_2211_08770_gb300 import build
    build.build()
    monkeypatch.setenv("TTGB_CHOL_NB", str(nb))
    c = T.Ctx(0, "fp64")
    rng = np.random.default_rng(3)
    X = rng.standard_normal((n, 2 * n + 60))
    for i, d in enumerate(dep):       # exactly dependent rows
        X[d] = X[3 + i] - 2 * X[7 + i] if i % 2 == 0 else X[10 + i]
    G = X @ X.T
    Gd = torch.tensor(G, device="cuda")
    L = torch.empty_like(Gd)
    Ti = torch.empty_like(Gd)
    nd = T.tt_cholesky_inverse(c, n, Gd.data_ptr(), L.data_ptr(), Ti.data_ptr(), 0.0, 1e-12)
    assert nd == len(dep)
    Lh, Th = L.cpu().numpy(), Ti.cpu().numpy()
    for d in dep:
        assert np.all(Lh[:, d] == 0) and np.all(Th[d] == 0) and np.all(Th[:, d] == 0)
    assert np.linalg.norm(Lh @ Lh.T - G) <= 1e-12 * np.linalg.norm(G)
    keep = [i for i in range(n) if i not in dep]
    Q = Th[keep] @ X
    assert np.allclose(Q @ Q.T, np.eye(n - len(dep)), atol=1e-10)
    c.close()


def test_tc_gram_bounded_wait_runs_out_and_context_recovers(ctx):
    # A one-cycle limit makes the row Gram's mbarrier waits give up before
    # the first TMA copy lands: the kernel records the timeout, lets its
    # issued copies land, waits for its MMAs, frees TMEM and returns; the
    # call reports TT_ERR_TIMEOUT.  With the default limit restored the same
    # context computes the Gram, and a TT-round on it succeeds.
    n, K = 256, 32768
    g = torch.Generator(device="cpu").manual_seed(99)
    Xh = torch.randn(n, K, generator=g, dtype=torch.float32)
    X = Xh.cuda()
    G = torch.zeros((n, n), device="cuda", dtype=torch.float32)
    ctx.set_tc_wait_limit(1)
    try:
        with pytest.raises(T.TTError) as e:
            T.tt_gram_f32(ctx, n, K, X.data_ptr(), K, G.data_ptr(), True)
        assert e.value.name == "TT_ERR_TIMEOUT"
    finally:
        ctx.set_tc_wait_limit(0)
    T.tt_gram_f32(ctx, n, K, X.data_ptr(), K, G.data_ptr(), True)
    torch.cuda.synchronize()
    Xd = Xh.numpy().astype(np.float64)
    ref = Xd @ Xd.T
    mask = _lower_tiles_mask(n, 128)
    dg = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert (np.abs(G.cpu().numpy().astype(np.float64) - ref)[mask] / dg[mask]).max() <= 4e-3
    with pytest.raises(T.TTError):
        ctx.set_tc_wait_limit(-1)
    import oracle as O
    from ttinputs import random_tts
    x = O.tt_add([1.0, -0.5], random_tts(5, 2, 4, 64, 24))
    y, _ = T.tt_round(ctx, T.tt_tensor_create(ctx, x), 1e-6)
    assert O.tt_diff_norm(y.cores(), x) <= 2e-6 * O.tt_norm(x)
