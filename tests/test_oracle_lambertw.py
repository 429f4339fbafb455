"""Pins for the oracle's principal-branch Lambert W0 (named by Eq. 1 and Eq. 13).

Independent checks: scipy's lambertw (a library routine), the defining
residual, special values, and the forward conformal map of the grating cloak
(z = w + i A exp(i k w), whose v = 0 line is Eq. 2), under which
W0(zeta(z)) = -kA exp(i k w) exactly."""
import math

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")


def test_w0_matches_scipy_on_grid(orc):
    r = np.concatenate([np.geomspace(1e-8, 0.3, 25), np.linspace(0.3, 6.0, 40)])
    th = np.linspace(-math.pi, math.pi, 73)
    z = (r[:, None] * np.exp(1j * th[None, :])).ravel()
    # keep away from the branch cut (-inf, -1/e] where W0 is discontinuous
    near_cut = (np.abs(z.imag) < 1e-2) & (z.real < -1 / math.e + 1e-3)
    z = z[~near_cut]
    w, it = orc.lambertw0(z)
    ref = scipy_special.lambertw(z, 0)
    err = np.abs(w - ref) / np.maximum(np.abs(ref), 1e-300)
    assert err.max() < 5e-14, (z[err.argmax()], w[err.argmax()], ref[err.argmax()])
    assert it.max() < 30


def test_w0_residual(orc):
    rng = np.random.default_rng(7)
    z = rng.uniform(-0.6, 0.6, 2000) + 1j * rng.uniform(-0.6, 0.6, 2000)
    z = z[~((np.abs(z.imag) < 1e-3) & (z.real < -1 / math.e))]
    w, _ = orc.lambertw0(z)
    res = np.abs(w * np.exp(w) - z)
    assert (res <= 4e-16 * np.maximum(np.abs(z), 1e-300) + 1e-300).all() or res.max() < 1e-15


def test_w0_special_values(orc):
    omega = 0.5671432904097838729999686622  # the omega constant, W0(1)
    w, _ = orc.lambertw0([1.0, math.e, -1 / math.e, 0.0, -math.exp(-1.0) * 1.0])
    assert abs(w[0] - omega) < 1e-15
    assert abs(w[1] - 1.0) < 1e-15
    assert abs(w[2] + 1.0) < 1e-7          # branch point: W0(-1/e) = -1 (square-root sensitivity)
    assert w[3] == 0
    t = np.linspace(-0.99, 5.0, 200)
    wt, _ = orc.lambertw0(t * np.exp(t))
    assert np.abs(wt - t).max() < 1e-12
    assert np.abs(wt.imag).max() == 0.0 or np.abs(wt.imag).max() < 1e-300


def test_w0_forward_map_identity(orc):
    """For w = u + i v above the virtual mirror (v >= 0), z = w + i A e^{ikw}
    is the physical point; W0(zeta(z)) must equal -kA e^{ikw}."""
    from paper_1012_5107_gb300 import inputs
    for lam, A in [(1.0, 0.04), (1.0, 3 / (16 * math.pi)), (0.7, 0.05)]:
        sc = orc.Scene(inputs.base_scene(Lambda=lam, A=A))
        k = 2 * math.pi / lam
        rng = np.random.default_rng(11)
        w = rng.uniform(-3 * lam, 3 * lam, 500) + 1j * rng.uniform(0.0, 1.5 * lam, 500)
        z = w + 1j * A * np.exp(1j * k * w)
        out = orc.index(sc, z.real, z.imag)
        W = out[:, 0] + 1j * out[:, 1]
        expect = -k * A * np.exp(1j * k * w)
        assert np.abs(W - expect).max() < 2e-15 * max(1.0, k * A) * 4
