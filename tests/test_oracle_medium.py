"""Pins for the oracle's index profile (Eq. 1), gradient (Eq. 12) and the
trochoid grating (Eqs. 2-3)."""
import json
import math
import os

import numpy as np

from paper_1012_5107_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _sc(orc, **kw):
    return orc.Scene(inputs.base_scene(**kw))


def test_gradient_eq12_matches_finite_differences(orc):
    for A in (0.04, 3 / (16 * math.pi)):
        sc = _sc(orc, A=A)
        rng = np.random.default_rng(3)
        x = rng.uniform(-2, 2, 300)
        xi = orc.trochoid(sc, x)
        y = xi[:, 1] + rng.uniform(0.01, 1.5, 300)      # above the grating
        h = 1e-6
        n = lambda xx, yy: orc.index(sc, xx, yy)[..., 2]
        fdx = (n(x + h, y) - n(x - h, y)) / (2 * h)
        fdy = (n(x, y + h) - n(x, y - h)) / (2 * h)
        g = orc.index(sc, x, y)
        scale = np.maximum(1.0, np.abs(g[:, 3]) + np.abs(g[:, 4]))
        assert np.abs(g[:, 3] - fdx).max() / scale.max() < 1e-8
        assert np.abs(g[:, 4] - fdy).max() / scale.max() < 1e-8
        assert (g[:, 5] == 0).all()                     # z-invariance (Sec. 3)


def test_index_on_surface_closed_form(orc):
    """On the grating (Eq. 2, parameter xi) the index is 1/|1 - kA e^{ik xi}|."""
    A = 0.05
    sc = _sc(orc, A=A)
    k = 2 * math.pi
    xi = np.linspace(-1.5, 1.5, 301)
    x = xi - A * np.sin(k * xi)
    y = A * np.cos(k * xi)
    n = orc.index(sc, x, y)[:, 2]
    expect = 1 / np.abs(1 - k * A * np.exp(1j * k * xi))
    assert np.abs(n - expect).max() < 1e-13


def test_paper_printed_index_values(orc):
    """Fig. 1(a): Lambda = 1, A = 3/(16 pi) gives n_min = 0.727 and n/n_min
    spanning [1.0, 2.2]; Fig. 5 prints 1/n_min = 1.37."""
    gv = json.load(open(GOLDEN))["grating_fig1a"]
    A = gv["A_over_pi"] / math.pi
    assert abs(A - gv["A_approx"]) < 0.005
    sc = _sc(orc, A=A)
    # index along the grating surface and over the cloak above it
    xi = np.linspace(0, 1, 2001)
    xs = xi - A * np.sin(2 * math.pi * xi)
    ys = A * np.cos(2 * math.pi * xi)
    n_s = orc.index(sc, xs, ys)[:, 2]
    xg, yg = np.meshgrid(np.linspace(0, 1, 101), np.linspace(0, 1.1, 111))
    ok = yg > orc.trochoid(sc, xg.ravel())[:, 1].reshape(xg.shape)
    n_g = orc.index(sc, xg[ok], yg[ok])[:, 2]
    n_all = np.concatenate([n_s, n_g])
    n_min, n_max = n_all.min(), n_all.max()
    tol = gv["print_tolerance"]
    assert abs(n_min - gv["n_min"]) < tol
    assert abs(n_min - gv["n_min_fig3"]) < tol
    assert abs(1 / n_min - gv["inv_n_min"]) < 0.01
    lo, hi = gv["n_ratio_range"]
    assert abs(n_max / n_min - hi) < 0.01
    assert abs(n_all.max() / n_min - hi) < 0.01 and n_all.min() / n_min >= lo - 1e-12
    # the exact extremes: troughs 1/(1+kA), crests 1/(1-kA)
    kA = 2 * math.pi * A
    assert abs(n_min - 1 / (1 + kA)) < 1e-12
    assert abs(n_max - 1 / (1 - kA)) < 1e-12


def test_index_tends_to_one_far_above(orc):
    sc = _sc(orc, A=0.04)
    k, kA = 2 * math.pi, 2 * math.pi * 0.04
    for y in (1.0, 2.0, 3.0):
        x = np.linspace(0, 1, 17)
        n = orc.index(sc, x, np.full_like(x, y))[:, 2]
        lead = kA * math.exp(-k * y)
        # 1/|1+W| with W ~ zeta: n - 1 ~ -Re(zeta) = kA e^{-ky} cos(kx)
        assert np.abs(n - 1 - lead * np.cos(k * x)).max() < 3 * lead * lead + 1e-15


def test_virtual_mirror_is_the_trochoid(orc):
    """v = y + Re(W0)/k vanishes on the Eq. 2 curve and is positive above it."""
    A = 0.06
    sc = _sc(orc, A=A)
    k = 2 * math.pi
    xi = np.linspace(-1, 1, 401)
    x = xi - A * np.sin(k * xi)
    y = A * np.cos(k * xi)
    W = orc.index(sc, x, y)
    v = y + W[:, 0] / k
    assert np.abs(v).max() < 1e-15
    W2 = orc.index(sc, x, y + 0.01)
    assert ((y + 0.01 + W2[:, 0] / k) > 0).all()


def test_explicit_form_eq3_matches_parametric_eq2(orc):
    for A in (0.04, 0.06, 0.1):
        sc = _sc(orc, A=A)
        lam = 1.0
        yv = np.linspace(-A * 0.999, A * 0.999, 101)
        base = lam / (2 * math.pi) * np.arccos(yv / A) - np.sqrt(A * A - yv * yv)   # Eq. 3
        for N in (-2, 0, 3):
            for sign in (+1, -1):
                x = sign * base + N * lam
                ys = orc.trochoid(sc, x)[:, 1]
                assert np.abs(ys - yv).max() < 1e-14


def test_kepler_exact_at_half_periods(orc):
    sc = _sc(orc, A=0.06)
    x = np.arange(-6, 7) * 0.5
    xi = orc.trochoid(sc, x)[:, 0]
    assert (np.abs(xi - x) <= 8 * np.finfo(float).eps * np.maximum(1.0, np.abs(x))).all()


def test_normal_from_eq2_tangent_equals_gradient_of_v(orc):
    """Two independent normals: the tangent of Eq. 2 and grad v / |grad v| =
    (Im 1/(1+W0), Re 1/(1+W0)) / n."""
    A = 0.05
    sc = _sc(orc, A=A)
    x = np.linspace(-1, 1, 211)
    t = orc.trochoid(sc, x)
    W = orc.index(sc, x, t[:, 1])
    r = 1 / (1 + W[:, 0] + 1j * W[:, 1])
    g = np.stack([r.imag, r.real], -1)
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    assert np.abs(g - t[:, 2:4]).max() < 1e-12
