"""The cross-correlation function C(di, dj) (Eq. 15 over shifts, Sec. 5) on
the GPU against the oracle: every shift of small maps, sampled shifts at the
benchmark's image size, the peak and the mean over reference pairs, and the
rejected arguments."""
import numpy as np
import pytest

from paper_1012_5107_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5      # C is dimensionless; the bar for cross-correlations is 1e-4


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


def _img(seed, H, W, C=3):
    return np.random.default_rng(seed).random((H, W, C)).astype(np.float32)


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("H,W,C,fov,mdi,mdj", [
    (50, 70, 3, 50.0, 5, 9),      # ragged sizes, tiles only partly used
    (33, 41, 1, 25.0, 0, 12),     # one channel, column shifts only
    (17, 200, 3, 10.0, 9, 3),     # shifts larger than the window in rows
    (64, 64, 4, 50.0, 40, 40),    # more shifts than pixels in the window overlap
])
def test_map_matches_oracle(rt, orc, H, W, C, fov, mdi, mdj):
    f, g = _img(1, H, W, C), _img(2, H, W, C)
    g = (0.5 * f + 0.5 * g).astype(np.float32)
    m, pk = rt.xcorr_map([(_cuda(f), _cuda(g))], fov, 50.0, mdi, mdj)
    j0, j1 = orc.fov_columns(W, 50.0, fov)
    o = orc.xcorr_map(f, g, j0, j1, mdi, mdj)
    m = m.cpu().numpy()
    assert m.shape == o.shape
    assert np.abs(m - o).max() < TOL
    p = pk.cpu().numpy()
    k = np.argmax(o[..., C])
    assert abs(p[0] - o[..., C].ravel()[k]) < TOL
    assert (int(p[1]), int(p[2])) == (k // (2 * mdj + 1) - mdi, k % (2 * mdj + 1) - mdj)


def test_peak_finds_the_shift(rt):
    rng = np.random.default_rng(3)
    H, W, si, sj = 96, 128, -4, 7
    big = rng.random((H + 40, W + 40, 3)).astype(np.float32)
    f = big[20:20 + H, 20:20 + W]
    g = big[20 - si:20 - si + H, 20 - sj:20 - sj + W]
    _, pk = rt.xcorr_map([(_cuda(f), _cuda(g))], 50.0, 50.0, 16, 16)
    p = pk.cpu().numpy()
    assert (int(p[1]), int(p[2])) == (si, sj)
    assert p[0] > 0.8


def test_mean_over_reference_pairs(rt, orc):
    pairs = [(_img(10 + q, 40, 48), _img(20 + q, 40, 48)) for q in range(3)]
    pairs = [(f, (0.7 * f + 0.3 * g).astype(np.float32)) for f, g in pairs]
    m, _ = rt.xcorr_map([(_cuda(f), _cuda(g)) for f, g in pairs], 50.0, 50.0, 4, 6)
    o = np.mean([orc.xcorr_map(f, g, 0, 48, 4, 6) for f, g in pairs], axis=0)
    assert np.abs(m.cpu().numpy() - o).max() < TOL


def test_zero_shift_is_c00(rt):
    import torch
    f, g = _img(30, 60, 80), _img(31, 60, 80)
    tf, tg = _cuda(f), _cuda(g)
    m, _ = rt.xcorr_map([(tf, tg)], 25.0, 50.0, 0, 0)
    c = rt.xcorr(tf, tg, [25.0], 50.0)
    torch.cuda.synchronize()
    assert np.abs(m.cpu().numpy()[0, 0] - c.cpu().numpy()[0]).max() < 1e-6


def test_renders_at_benchmark_size(rt, orc):
    """The cloaked and flat-mirror renders of the 512 x 512 x 4 workload (FP32
    path): a +-32 shift map, checked against the oracle on the central shifts."""
    import torch
    imgs = {}
    for kind in ("mirror", "cloak"):
        sc = rt.Scene(inputs.three_renders(inputs.config_main(precision=0))[kind])
        imgs[kind] = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
        sc.render(imgs[kind])
    torch.cuda.synchronize()
    m, pk = rt.xcorr_map([(imgs["mirror"], imgs["cloak"])], 50.0, 50.0, 32, 32)
    m = m.cpu().numpy()
    f, g = imgs["mirror"].cpu().numpy(), imgs["cloak"].cpu().numpy()
    j0, j1 = orc.fov_columns(512, 50.0, 50.0)
    o = orc.xcorr_map(f, g, j0, j1, 2, 2)
    assert np.abs(m[30:35, 30:35] - o).max() < TOL
    assert np.isfinite(m).all()
    p = pk.cpu().numpy()
    assert p[0] >= m[32, 32, 3] - 1e-12


@pytest.mark.parametrize("over,msg", [
    (dict(max_di=65), "max_di"), (dict(fov=0.0), "no pixel column"), (dict(n=65), "n_pairs"),
])
def test_rejected_arguments(rt, over, msg):
    f = _cuda(_img(40, 16, 16))
    pairs = [(f, f)] * over.get("n", 1)
    with pytest.raises(rt.RtError) as e:
        rt.xcorr_map(pairs, over.get("fov", 50.0), 50.0, over.get("max_di", 2), 2)
    assert e.value.code == rt.RT_EINVAL and msg in str(e.value)
