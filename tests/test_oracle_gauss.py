"""Pins for the oracle's Gaussian conformal cloak (Sec. 2, Eq. 5, Fig. 1(b),
Fig. 4): the Faddeeva function against library routines, the index range the
paper prints for w = 0.306, h = 0.13, the shallow-bump limit of Eq. 5, the
inverse map, the index gradient, the bump surface and its line hits, and the
2-D exactness of the cloak."""
import math

import numpy as np
import pytest

from paper_1012_5107_gb300 import inputs

special = pytest.importorskip("scipy.special")


def _sc(orc, **kw):
    return orc.Scene(inputs.gauss_scene(**kw))


# ---------------------------------------------------------------------------
# Faddeeva function F(s) = exp(-s^2) erfc(-i s)
# ---------------------------------------------------------------------------
def test_faddeeva_matches_library(orc):
    s = np.linspace(-20, 20, 401)[None, :] + 1j * np.linspace(-0.5, 6.0, 131)[:, None]
    ref = special.wofz(s)
    got = orc.faddeeva(s)
    err = np.abs(got - ref)
    assert err.max() < 1e-14
    assert (err / np.abs(ref)).max() < 1e-13


def test_faddeeva_on_the_axes(orc):
    x = np.linspace(-12, 12, 2401)
    f = orc.faddeeva(x + 0j)
    assert np.abs(f.real - np.exp(-x * x)).max() < 2e-15
    assert np.abs(f.imag - 2 / math.sqrt(math.pi) * special.dawsn(x)).max() < 2e-15
    y = np.linspace(0, 30, 601)
    g = orc.faddeeva(1j * y)
    assert np.abs(g.imag).max() < 1e-15
    assert np.abs(g.real / special.erfcx(y) - 1).max() < 1e-13
    assert abs(orc.faddeeva(np.array([0j]))[0] - 1.0) < 1e-15


# ---------------------------------------------------------------------------
# The map z(w) = w + i h F(w / w_b) and the index n = |dw/dz|
# ---------------------------------------------------------------------------
def test_index_range_of_fig1b(orc):
    """w = 0.306, h = 0.13: n_min = 0.873 and n/n_min spans [1, 2.2]
    (Fig. 1(b)).  n = 1/|z'| takes its extremes on the bump (v = 0)."""
    sc = _sc(orc)
    u = np.linspace(-3, 3, 60001)
    _, dz = orc.gauss_map(sc, u + 0j)
    n = 1 / np.abs(dz)
    assert round(n.min(), 3) == 0.873
    assert round(n.max() / n.min(), 1) == 2.2
    # inside the cloak region n stays within the range taken on the bump
    xs, ys = np.meshgrid(np.linspace(-2, 2, 201), np.linspace(0, 1.1, 111))
    r = orc.index(sc, xs.ravel(), ys.ravel())
    above = r[:, 1] >= 0
    assert r[above, 2].min() >= n.min() - 1e-12 and r[above, 2].max() <= n.max() + 1e-12
    # and tends to 1 far from the bump: z' ~ 1 + h w_b / (sqrt(pi) z^2)
    for zf in (40j, 40.0 + 0.5j, -25.0 + 10j):
        far = orc.index(sc, zf.real, zf.imag)[2]
        pred = 1 / abs(1 + 0.13 * 0.306 / (math.sqrt(math.pi) * zf * zf))
        assert abs((far - 1) / (pred - 1) - 1) < 0.01


def test_zero_height_is_the_identity_map(orc):
    """h = 0: the map is the identity, n = 1 and no force."""
    r = orc.index(_sc(orc, A=0.0), np.array([0.3, -1.0]), np.array([0.5, 2.0]))
    assert np.abs(r[:, 2] - 1).max() == 0 and np.abs(r[:, 3:]).max() == 0
    assert np.abs(r[:, 0] - [0.3, -1.0]).max() == 0 and np.abs(r[:, 1] - [0.5, 2.0]).max() == 0


def test_shallow_bump_limit_is_eq5(orc):
    """The bump (the image of v = 0) tends to y = h exp(-(x/w)^2) (Eq. 5) with
    an error of second order in h."""
    x = np.linspace(-1.5, 1.5, 301)
    errs = []
    for h in (2e-3, 1e-3):
        sc = _sc(orc, A=h)
        y = orc.surface(sc, x)[:, 0]
        errs.append(np.abs(y - h * np.exp(-(x / 0.306) ** 2)).max())
        assert errs[-1] < 3 * h * h / 0.306
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_inverse_map_round_trip(orc):
    sc = _sc(orc)
    xs, ys = np.meshgrid(np.linspace(-4, 4, 161), np.linspace(0, 1.1, 56))
    r = orc.index(sc, xs.ravel(), ys.ravel())
    above = r[:, 1] >= 0
    w = r[above, 0] + 1j * r[above, 1]
    z, _ = orc.gauss_map(sc, w)
    assert np.abs(z - (xs.ravel() + 1j * ys.ravel())[above]).max() < 1e-14
    # far field: z - w = i h F(w/w_b) ~ -h w_b / (sqrt(pi) w)
    zf = np.array([30.0 + 5j, -25.0 + 40j])
    rf = orc.index(sc, zf.real, zf.imag)
    wf = rf[:, 0] + 1j * rf[:, 1]
    assert np.abs((zf - wf) / (-0.13 * 0.306 / (math.sqrt(math.pi) * wf)) - 1).max() < 1e-3


def test_index_gradient_matches_finite_differences(orc):
    sc = _sc(orc)
    rng = np.random.default_rng(7)
    pts = np.stack([rng.uniform(-1, 1, 40), rng.uniform(0.15, 1.0, 40)], -1)
    d = 1e-6
    for x, y in pts:
        g = orc.index(sc, x, y)
        fx = (orc.index(sc, x + d, y)[2] - orc.index(sc, x - d, y)[2]) / (2 * d)
        fy = (orc.index(sc, x, y + d)[2] - orc.index(sc, x, y - d)[2]) / (2 * d)
        assert abs(g[3] - fx) < 1e-7 * max(1, abs(fx)) and abs(g[4] - fy) < 1e-7 * max(1, abs(fy))
        assert g[5] == 0.0


# ---------------------------------------------------------------------------
# The bump surface
# ---------------------------------------------------------------------------
def test_event_function_vanishes_on_the_bump(orc):
    """v = Im w is zero on the bump's parametric form x = u - h Im F(u/w_b),
    y = h exp(-(u/w_b)^2) and positive above it."""
    sc = _sc(orc)
    u = np.linspace(-2, 2, 81)
    s = u / 0.306
    x = u - 0.13 * 2 / math.sqrt(math.pi) * special.dawsn(s)
    y = 0.13 * np.exp(-s * s)
    r = orc.index(sc, x, y)
    assert np.abs(r[:, 1]).max() < 1e-14
    assert np.abs(r[:, 0] - u).max() < 1e-13
    assert np.all(orc.index(sc, x, y + 1e-3)[:, 1] > 0)
    # the surface helper gives the same heights
    assert np.abs(orc.surface(sc, x)[:, 0] - y).max() < 1e-14


def test_surface_slope_and_normal(orc):
    sc = _sc(orc)
    x = np.linspace(-1.2, 1.2, 49)
    d = 1e-6
    s = orc.surface(sc, x)
    fd = (orc.surface(sc, x + d)[:, 0] - orc.surface(sc, x - d)[:, 0]) / (2 * d)
    assert np.abs(s[:, 1] - fd).max() < 1e-8
    # the normal is the unit upward normal of the tangent (1, slope)
    assert np.abs(s[:, 2] + s[:, 1] * s[:, 3]).max() < 1e-14
    assert np.abs(np.hypot(s[:, 2], s[:, 3]) - 1).max() < 1e-15 and np.all(s[:, 3] > 0)


def test_line_hit_against_dense_sampling(orc):
    sc = _sc(orc, A=0.2, gauss_w=0.3)
    rng = np.random.default_rng(11)
    for _ in range(40):
        X = np.array([rng.uniform(-1.5, 1.5), rng.uniform(0.3, 2.0), 0.2])
        ang = rng.uniform(-85, -10)
        p = np.array([math.cos(math.radians(ang)), math.sin(math.radians(ang)), 0.1])
        p /= np.linalg.norm(p)
        t = orc.surface_line_hit(sc, X, p)
        ts = np.linspace(0, (X[1] + 1e-9) / -p[1], 20001)
        h = X[1] + ts * p[1] - orc.surface(sc, X[0] + ts * p[0])[:, 0]
        k = int(np.argmax(h <= 0))
        assert h[k] <= 0 and np.all(h[:k] > 0)
        assert ts[k - 1] - 1e-12 <= t <= ts[k] + 1e-12
        assert abs(X[1] + t * p[1] - orc.surface(sc, X[0] + t * p[0])[0, 0]) < 1e-12


# ---------------------------------------------------------------------------
# 2-D exactness (Sec. 5): in virtual space the rays are straight lines
# reflected at v = 0
# ---------------------------------------------------------------------------
def test_2d_gaussian_cloak_is_a_flat_mirror_in_virtual_space(orc):
    sc = _sc(orc, H=6.0, E=1000.0, integrator=1, rtol=1e-12, atol=1e-12)
    for x0, ang in ((0.9, -40.0), (0.1, -60.0), (-0.4, -85.0)):
        X = np.array([x0, 5.5, 0.0])
        n = orc.index(sc, X[0], X[1])[2]
        p = n * np.array([math.cos(math.radians(ang)), math.sin(math.radians(ang)), 0.0])
        rec, traj = orc.trace_from(sc, X, p, medium=1, traj_cap=20000)
        assert rec["bounces"] == 1 and rec["status"] == 0
        W = orc.index(sc, traj[:, 0], traj[:, 1])
        w = W[:, 0] + 1j * W[:, 1]
        ih = int(np.argmin(np.abs(w.imag)))
        assert abs(w[ih].imag) < 1e-12
        # the virtual direction is the physical one turned by g = dw/dz = 1/z'(w)
        _, dz0 = orc.gauss_map(sc, w[:1])
        d_in = (p[0] + 1j * p[1]) / dz0[0]
        d_in /= abs(d_in)
        d_out = d_in.conjugate()
        dist_pre = np.abs(((w[: ih + 1] - w[0]) * d_in.conjugate()).imag)
        dist_post = np.abs(((w[ih:] - w[ih]) * d_out.conjugate()).imag)
        assert dist_pre.max() < 1e-9 and dist_post.max() < 1e-9, (dist_pre.max(), dist_post.max())


def test_invalid_gaussian_scenes(orc):
    for bad in (dict(gauss_w=0.0), dict(A=0.3, gauss_w=0.306), dict(flags=orc.FLAG_FRESNEL)):
        with pytest.raises(ValueError):
            orc.render_pixels(orc.Scene(inputs.gauss_scene(**bad)), [0])


def test_renders_converge_and_far_rays_see_a_flat_mirror(orc):
    """Cloaked-bump render: RK4 at h = Lambda/200 agrees with tight
    Dormand-Prince; in the bare-bump render the rays that reflect far from
    the bump (|x| > 8 w) leave as from the flat mirror."""
    base = inputs.gauss_scene(width=24, height=24, spp=1, precision=1)
    pix = np.arange(24 * 24)
    _, r4 = orc.render_pixels(orc.Scene(base), pix, records=True)
    _, rd = orc.render_pixels(orc.Scene(dict(base, integrator=1, rtol=1e-10, atol=1e-10)), pix, records=True)
    same = (r4["bounces"] == rd["bounces"]) & (r4["status"] == rd["status"])
    assert same.mean() > 0.97
    assert np.abs(r4["dir"] - rd["dir"])[same].max() < 1e-7
    bare = dict(base, cloak=0)
    _, rb = orc.render_pixels(orc.Scene(bare), pix, records=True)
    _, rf = orc.render_pixels(orc.Scene(dict(bare, mirror=0)), pix, records=True)
    far = (rb["bounces"] == 1) & (np.abs(rb["pos"][:, 0]) > 8 * 0.306)
    assert far.sum() > 100
    assert np.abs(rb["dir"][far] - rf["dir"][far]).max() < 1e-12
    assert np.abs(rb["pos"][far] - rf["pos"][far]).max() < 1e-12
