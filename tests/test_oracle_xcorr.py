"""Pins for the oracle's image cross-correlation (Sec. 5, Eqs. 14-15)."""
import json
import os

import numpy as np

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _img(seed, H=40, W=50, C=3):
    rng = np.random.default_rng(seed)
    return rng.random((H, W, C)).astype(np.float32)


def test_identities_from_sec5(orc):
    f = _img(1)
    W = f.shape[1]
    gv = GOLD["xcorr_identities"]
    assert np.allclose(orc.xcorr(f, f, 0, W), gv["identical"], atol=1e-12)
    for a in (0.25, 0.7, 1.0):
        g = (a * f.astype(np.float64)).astype(np.float32)
        assert np.allclose(orc.xcorr(f, g, 0, W), a, atol=1e-6)
    comp = (1.0 - f).astype(np.float32)
    assert np.allclose(orc.xcorr(f, comp, 0, W), gv["complement"], atol=1e-6)
    shifted = (f + 0.3).astype(np.float32)               # mean subtraction (Eq. 14)
    assert np.allclose(orc.xcorr(f, shifted, 0, W), 1.0, atol=1e-6)
    other = _img(2)
    assert np.abs(orc.xcorr(f, other, 0, W)).max() < 0.1


def test_normalised_by_reference_energy_only(orc):
    """Eq. 15 divides by the reference's energy alone, so C(f, 2f) = 2 (not a
    Pearson coefficient, which would be 1)."""
    f = _img(3)
    g = (2.0 * f.astype(np.float64)).astype(np.float32)
    assert np.allclose(orc.xcorr(f, g, 0, f.shape[1]), 2.0, atol=1e-6)
    assert np.allclose(orc.xcorr(g, f, 0, f.shape[1]), 0.5, atol=1e-6)


def test_window_and_stacked_channels(orc):
    f = _img(4)
    g = _img(5)
    g[:, 10:20] = f[:, 10:20]
    assert np.allclose(orc.xcorr(f, g, 10, 20), 1.0, atol=1e-12)
    out = orc.xcorr(f, g, 0, 50)
    num = den = 0.0
    for c in range(3):
        a = f[..., c] - f[..., c].astype(np.float64).mean()
        b = g[..., c] - g[..., c].astype(np.float64).mean()
        num += (a * b).sum(); den += (a * a).sum()
    assert abs(out[3] - num / den) < 1e-12


def test_fov_columns(orc):
    assert orc.fov_columns(512, 50.0, 50.0) == (0, 512)
    assert orc.fov_columns(511, 50.0, 0.0) == (255, 256)
    assert orc.fov_columns(512, 50.0, 0.0) == (0, 0)
    j0, j1 = orc.fov_columns(512, 50.0, 10.0)
    assert j1 - j0 < 512 and j0 + j1 == 512
    j0b, j1b = orc.fov_columns(512, 50.0, 25.0)
    assert j0b < j0 and j1b > j1
    assert orc.fov_columns(1, 50.0, 0.0) == (0, 1)
