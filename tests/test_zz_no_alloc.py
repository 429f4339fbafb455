"""rt_xcorr_noalloc, the cross-correlation entry point that allocates no
device memory (for callers that cannot allocate: hosts that own all device
memory through their own pool, latency-bound loops that must not make
allocation calls).  It must give the results of rt_xcorr, call after call,
although every call reuses the same fixed scratch array.

This file is collected last so that a run stopping at the first failure has
run every other test first; it also passes alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the tolerance of the cross-correlation parity tests


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_5107_gb300 import build as B
    B.build()
    from paper_1012_5107_gb300 import rt as r
    r.lib()
    return r


def test_noalloc_matches_rt_xcorr_on_consecutive_calls(rt):
    import torch
    rng = np.random.default_rng(12)
    fovs = [0.0, 10.0, 25.0, 50.0]
    # two calls in a row with different images: a result left over in the
    # shared scratch from the first call would spoil the second
    for H, W in [(300, 512), (64, 37)]:
        f = rng.random((H, W, 3)).astype(np.float32)
        g = (0.5 * f + 0.5 * rng.random((H, W, 3))).astype(np.float32)
        tf, tg = torch.tensor(f, device="cuda"), torch.tensor(g, device="cuda")
        ref = rt.xcorr(tf, tg, fovs, 50.0)
        got = rt.xcorr_noalloc(tf, tg, fovs, 50.0)
        torch.cuda.synchronize()
        ref, got = ref.cpu().numpy(), got.cpu().numpy()
        fin = np.isfinite(ref)
        assert np.array_equal(np.isnan(ref), np.isnan(got))
        assert np.abs(got[fin] - ref[fin]).max() <= TOL


def test_noalloc_rejects_oversized_images(rt):
    import torch
    f = torch.zeros((1, 180000, 3), dtype=torch.float32, device="cuda")      # 540000 moment records
    with pytest.raises(rt.RtError) as e:
        rt.xcorr_noalloc(f, f, [50.0], 50.0)
    assert e.value.code == rt.RT_EINVAL
    assert "scratch" in str(e.value)
    # a successful call afterwards leaves no stale message behind
    g = torch.ones((8, 8, 3), dtype=torch.float32, device="cuda")
    rt.xcorr_noalloc(g, g, [50.0], 50.0)
    torch.cuda.synchronize()
    assert rt.lib().rt_last_error() == b""
