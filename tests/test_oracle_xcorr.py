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


# ---------------------------------------------------------------------------
# The cross-correlation function C(di, dj) (Eq. 15 with shifts, Sec. 5)
# ---------------------------------------------------------------------------
def test_map_identities_at_zero_shift(orc):
    """At zero shift the map is C(0,0): the Sec. 5 identities hold there."""
    f = _img(11)
    W = f.shape[1]
    m = orc.xcorr_map(f, f, 0, W, 3, 4)
    assert m.shape == (7, 9, 4)
    assert np.allclose(m[3, 4], 1.0, atol=1e-12)
    g = (0.6 * f.astype(np.float64)).astype(np.float32)
    assert np.allclose(orc.xcorr_map(f, g, 0, W, 2, 2)[2, 2], 0.6, atol=1e-6)
    comp = (1.0 - f).astype(np.float32)
    assert np.allclose(orc.xcorr_map(f, comp, 0, W, 2, 2)[2, 2], -1.0, atol=1e-6)


def test_shifted_copy_peaks_at_the_shift(orc):
    """An image shifted within the photographic plane correlates best at the
    shift (Sec. 5); with finite photographs the peak is the overlap's share."""
    rng = np.random.default_rng(12)
    H, W, si, sj = 48, 64, 3, -5
    big = rng.random((H + 20, W + 20, 3)).astype(np.float32)
    f = big[10:10 + H, 10:10 + W]
    g = big[10 - si:10 - si + H, 10 - sj:10 - sj + W]     # g(i + si, j + sj) = f(i, j)
    m = orc.xcorr_map(f, g, 0, W, 6, 8)
    di, dj = np.unravel_index(np.argmax(m[..., 3]), m[..., 3].shape)
    assert (di - 6, dj - 8) == (si, sj)
    overlap = (H - abs(si)) * (W - abs(sj)) / (H * W)
    assert abs(m[6 + si, 8 + sj, 3] - overlap) < 0.05
    assert m[6, 8, 3] < 0.2


def test_swap_symmetry(orc):
    """sum f'(x) g'(x + d) = sum g'(y) f'(y - d): C_fg(d) S_ff = C_gf(-d) S_gg,
    which checks the overlap region and the mean subtraction independently."""
    f, g = _img(13, 30, 41), _img(14, 30, 41)
    j0, j1 = 5, 37
    a = orc.xcorr_map(f, g, j0, j1, 4, 6)
    b = orc.xcorr_map(g, f, j0, j1, 4, 6)
    fw = f[:, j0:j1].astype(np.float64)
    gw = g[:, j0:j1].astype(np.float64)
    sff = ((fw - fw.mean(axis=(0, 1))) ** 2).sum(axis=(0, 1))
    sgg = ((gw - gw.mean(axis=(0, 1))) ** 2).sum(axis=(0, 1))
    for c in range(3):
        assert np.allclose(a[..., c] * sff[c], b[::-1, ::-1, c] * sgg[c], rtol=1e-10, atol=1e-10)


def test_periodic_pattern_has_repeated_maxima(orc):
    """A pattern periodic in x gives maxima of C at multiples of its period (Sec. 5)."""
    H, W, P = 32, 60, 6
    jj = np.arange(W)
    row = (np.sin(2 * np.pi * jj / P) + 1.0) * 0.5
    f = np.repeat(row[None, :], H, axis=0).astype(np.float32)[..., None]
    m = orc.xcorr_map(f, f, 0, W, 0, 14)[0, :, 1]
    peaks = [d - 14 for d in range(1, 28) if m[d] > m[d - 1] and m[d] >= m[d + 1]]
    assert peaks == [-12, -6, 0, 6, 12]
    # a shift by a whole period loses only the columns that leave the window
    assert abs(m[14 + P] - (W - P) / W) < 0.02


def test_map_matches_c00_and_unrelated_images(orc):
    f, g = _img(15), _img(16)
    W = f.shape[1]
    m = orc.xcorr_map(f, g, 3, W - 3, 2, 3)
    assert np.allclose(m[2, 3], orc.xcorr(f, g, 3, W - 3), atol=1e-12)
    assert np.abs(m).max() < 0.1                         # unrelated images: near 0 everywhere
