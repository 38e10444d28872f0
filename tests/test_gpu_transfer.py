"""Host <-> device transfers of TT cores: the FP64 entry points (narrowed or
widened on the device for FP32 storage) and the storage-type entry points
(no conversion), from pageable and page-locked host memory."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
T = pytest.importorskip("paper_2211_08770_gb300.ttgb")

from ttinputs import random_tt  # noqa: E402


@pytest.fixture(scope="module")
def ctxs():
    from paper_2211_08770_gb300 import build
    build.build()
    out = {p: T.Ctx(0, p) for p in ("fp64", "mixed_tf32")}
    yield out
    for c in out.values():
        c.close()


def _cores():
    return random_tt(np.random.default_rng(5), [7, 33, 5, 64], [1, 6, 17, 9, 1])


@pytest.mark.parametrize("prec", ["fp64", "mixed_tf32"])
def test_fp64_entry_points_round_trip(ctxs, prec):
    # FP32 storage: the device narrowing and widening are round-to-nearest
    # conversions, the same as the host's
    c = ctxs[prec]
    x = _cores()
    got = T.tt_tensor_create(c, x).cores()
    for a, b in zip(got, x):
        want = b if prec == "fp64" else b.astype(np.float32).astype(np.float64)
        assert np.array_equal(a, want)


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "mixed_tf32"])
def test_storage_entry_points_round_trip(ctxs, prec, pinned):
    c = ctxs[prec]
    dt = np.float64 if prec == "fp64" else np.float32
    tdt = torch.float64 if prec == "fp64" else torch.float32
    x = [a.astype(dt) for a in _cores()]
    if pinned:
        hin = []
        for a in x:
            b = torch.empty(a.shape, dtype=tdt, pin_memory=True).numpy()
            b[...] = a
            hin.append(b)
        out = [torch.full((a.size + 3,), float("nan"), dtype=tdt, pin_memory=True).numpy() for a in x]
    else:
        hin = [a.copy() for a in x]
        out = [np.full(a.size + 3, np.nan, dtype=dt) for a in x]
    t = T.tt_tensor_create_storage(c, hin)
    views = t.download_storage(out)
    for v, a in zip(views, x):
        assert v.shape == a.shape and np.array_equal(v, a)
    # the FP64 reader sees the same values
    for g, a in zip(t.cores(), x):
        assert np.array_equal(g, a.astype(np.float64))
    with pytest.raises(ValueError):
        T.tt_tensor_create_storage(c, [a.astype(np.float16) for a in x])


@pytest.mark.parametrize("pinned", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "mixed_tf32"])
def test_round_to_host_matches_round_and_download(ctxs, prec, pinned):
    # the host copies made during the sweep equal the returned device result
    import oracle as O
    from ttinputs import coefficients, random_tts
    c = ctxs[prec]
    dt = np.float64 if prec == "fp64" else np.float32
    tdt = torch.float64 if prec == "fp64" else torch.float32
    xs = random_tts(31, 4, 6, 12, 5)
    x = O.tt_add(list(coefficients(32, 4)), xs)
    t = T.tt_tensor_create(c, x)
    _, n, r = t.shape()
    sizes = [r[k] * n[k] * r[k + 1] for k in range(len(n))]
    if pinned:
        out = [torch.full((m,), float("nan"), dtype=tdt, pin_memory=True).numpy() for m in sizes]
    else:
        out = [np.full(m, np.nan, dtype=dt) for m in sizes]
    y, err, views = T.tt_round_to_host(c, t, 1e-6, out)
    dev = y.download_storage([np.empty(m, dtype=dt) for m in sizes])
    for v, w in zip(views, dev):
        assert v.shape == w.shape and np.array_equal(v, w)
    assert O.tt_diff_norm([v.astype(np.float64) for v in views], x) <= (1e-6 + (1e-12 if prec == "fp64" else 1e-6)) * O.tt_norm(x)
    # d = 1 is a copy
    one = T.tt_tensor_create(c, [np.ascontiguousarray(x[0][:, :, :1])])
    y1, _, v1 = T.tt_round_to_host(c, one, 1e-6, [np.empty(n[0], dtype=dt) if not pinned else
                                                   torch.empty(n[0], dtype=tdt, pin_memory=True).numpy()])
    assert np.array_equal(v1[0].reshape(-1), x[0][:1, :, :1].reshape(-1).astype(dt))


def test_round_to_host_after_a_retried_rounding(monkeypatch):
    # a rounding redone after its series passes are judged invalid (forced)
    # still leaves the final result in the host buffers
    import oracle as O
    from ttinputs import coefficients, random_tts
    monkeypatch.setenv("TTGB_SERIES_PASS", "retry")
    c = T.Ctx(0, "mixed_tf32")
    try:
        x = O.tt_add(list(coefficients(34, 5)), random_tts(33, 5, 5, 16, 6))
        t = T.tt_tensor_create(c, x)
        _, n, r = t.shape()
        sizes = [r[k] * n[k] * r[k + 1] for k in range(len(n))]
        out = [torch.full((m,), float("nan"), dtype=torch.float32, pin_memory=True).numpy() for m in sizes]
        y, _, views = T.tt_round_to_host(c, t, 1e-6, out)
        assert c.stats()["series_retries"] == 1
        dev = y.download_storage([np.empty(m, dtype=np.float32) for m in sizes])
        for v, w in zip(views, dev):
            assert np.array_equal(v, w)
    finally:
        c.close()
