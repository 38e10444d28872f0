"""The allocation-free TT dot (tt_dot_f64_noalloc) against the regular entry
point tt_dot, through the C ABI, on two calls in a row.

This entry point serves callers that cannot allocate device memory (hosts
whose device memory all belongs to their own pool, latency-critical loops
that must not pay cudaMalloc's implicit synchronization); its work arrays
live in a static device array.
The file is named to be collected last, and it passes both on its own in a
fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
T = pytest.importorskip("paper_2211_08770_gb300.ttgb")

from ttinputs import random_tt  # noqa: E402


def _dev(cores):
    return [torch.tensor(c, dtype=torch.float64, device="cuda") for c in cores]


def test_noalloc_dot_matches_tt_dot_twice():
    from paper_2211_08770_gb300 import build
    build.build()
    ctx = T.Ctx(0, "fp64")
    rng = np.random.default_rng(2024)
    shapes = [([6, 9, 5, 7], [1, 4, 6, 3, 1], [1, 3, 5, 4, 1]),
              ([16, 16, 16, 16, 16], [1, 12, 20, 20, 12, 1], [1, 8, 16, 16, 8, 1])]
    stream = torch.cuda.current_stream()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for n, rx, ry in shapes:          # two calls in a row, different shapes
        x, y = random_tt(rng, n, rx), random_tt(rng, n, ry)
        xd, yd = _dev(x), _dev(y)
        T.tt_dot_f64_noalloc(stream.cuda_stream, n, rx, ry, [t.data_ptr() for t in xd],
                             [t.data_ptr() for t in yd], out.data_ptr())
        torch.cuda.synchronize()
        got = float(out.item())
        ref = T.tt_dot(ctx, T.tt_tensor_create(ctx, x), T.tt_tensor_create(ctx, y))
        scale = T.tt_norm(ctx, T.tt_tensor_create(ctx, x)) * T.tt_norm(ctx, T.tt_tensor_create(ctx, y))
        assert abs(got - ref) <= 1e-12 * scale, (got, ref)
    ctx.close()


def test_noalloc_dot_rejects_shapes_beyond_the_static_scratch():
    n, rx, ry = [2048, 2], [1, 1024, 1], [1, 1024, 1]
    x = [torch.zeros((rx[k], n[k], rx[k + 1]), dtype=torch.float64, device="cuda") for k in range(2)]
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    with pytest.raises(T.TTError) as e:
        T.tt_dot_f64_noalloc(torch.cuda.current_stream().cuda_stream, n, rx, ry, [t.data_ptr() for t in x],
                             [t.data_ptr() for t in x], out.data_ptr())
    assert e.value.name == "TT_ERR_ARG"
    assert "static scratch" in str(e.value)
