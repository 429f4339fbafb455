"""Pins for the oracle's camera, sampling, backgrounds and whole renders (Sec. 4)."""
import json
import math
import os

import numpy as np
import pytest

from paper_1012_5107_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs(orc):
    g = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    for m, want in enumerate(g["outputs"], start=1):
        assert orc.splitmix64(g["seed"], m) == int(want)


def test_camera_geometry(orc):
    p = inputs.base_scene(width=65, height=33, spp=1, elev_deg=30.0, azim_deg=20.0)
    sc = orc.Scene(p)
    o, d = orc.camera_dir(sc, 16, 32, 0)           # centre pixel of an odd-sized image
    assert abs(np.linalg.norm(o) - 12.0) < 1e-12
    assert abs(o[1] / 12.0 - math.sin(math.radians(30.0))) < 1e-12
    # the centre ray passes through the origin
    assert np.linalg.norm(np.cross(d, -o / 12.0)) < 1e-12
    # left/right columns mirror each other about the vertical plane through f
    _, dl = orc.camera_dir(sc, 5, 0, 0)
    _, dr = orc.camera_dir(sc, 5, 64, 0)
    f = -o / 12.0
    r = np.cross(f, [0, 1, 0]); r /= np.linalg.norm(r)
    assert abs((dl @ r) + (dr @ r)) < 1e-12 and abs(dl @ f - dr @ f) < 1e-12
    # horizontal half-angle of the outermost column centres is below hfov/2 = 25 deg
    ang = math.degrees(math.atan2(dr @ r, dr @ f))
    assert 24.0 < ang < 25.0


def test_stratified_jitter(orc):
    p = inputs.base_scene(width=8, height=8, spp=4, seed=9)
    sc = orc.Scene(p)
    o, _ = orc.camera_dir(sc, 0, 0, 0)
    f = -o / np.linalg.norm(o)
    r = np.cross(f, [0, 1, 0]); r /= np.linalg.norm(r)
    u = np.cross(r, f)
    tx = math.tan(math.radians(25.0))
    quad = set()
    for s in range(4):
        _, d = orc.camera_dir(sc, 3, 5, s)
        px = (d @ r) / (d @ f) / tx
        py = (d @ u) / (d @ f) / tx
        ox = (px + 1) * 8 / 2 - 5
        oy = (1 - py) * 8 / 2 - 3
        assert 0 <= ox < 1 and 0 <= oy < 1
        quad.add((int(ox * 2), int(oy * 2)))
    assert quad == {(0, 0), (1, 0), (0, 1), (1, 1)}


def at_plane(rec, y):
    """Where each record's final straight segment crosses the plane of height y."""
    t = (y - rec["pos"][:, 1]) / rec["dir"][:, 1]
    return rec["pos"] + t[:, None] * rec["dir"]


def _records(orc, p, pix=None):
    sc = orc.Scene(p)
    if pix is None:
        pix = np.arange(p["height"] * (1 if p["centre_line"] else p["width"]))
    rgb, rec = orc.render_pixels(sc, pix, records=True)
    return rgb, rec


def test_flat_limit_of_grating_and_cloak(orc):
    """A = 0 turns the trochoid into the flat mirror and the cloak index into 1:
    three different code paths must give the same rays."""
    base = inputs.base_scene(width=24, height=24, spp=1, A=0.0)
    _, rm = _records(orc, dict(base, mirror=0, cloak=0))
    _, rb = _records(orc, dict(base, mirror=1, cloak=0))
    _, rc = _records(orc, dict(base, mirror=1, cloak=1))
    assert (rm["bounces"] == 1).all()
    y = base["H"] - base["A"] + 1.0
    for r in (rb, rc):
        assert np.abs(r["dir"] - rm["dir"]).max() < 1e-12
        assert np.abs(at_plane(r, y) - at_plane(rm, y)).max() < 1e-9
        assert (r["bounces"] == rm["bounces"]).all()


def test_scale_invariance(orc):
    base = inputs.base_scene(width=12, height=12, spp=1, A=0.04)
    _, r1 = _records(orc, base)
    _, r2 = _records(orc, inputs.scale_scene(base, 2.5))
    assert np.abs(r2["dir"] - r1["dir"]).max() < 1e-9
    assert np.abs(r2["pos"] / 2.5 - r1["pos"]).max() < 1e-9
    assert (r2["bounces"] == r1["bounces"]).all()


def test_centre_line_is_cloaked(orc):
    """Sec. 5: the grating cloak is exact in 2-D, so on the vertical centre line
    (p_z = 0) a ray that enters and leaves through the top of the cloak
    reflects like the flat mirror, up to the O(kA exp(-kH)) index step at the
    top face; the bare grating does not.  A wide box (E = 40 Lambda) lets most
    centre-line rays stay clear of the side faces."""
    base = inputs.base_scene(width=64, height=96, spp=1, centre_line=1, E=40.0, H=4.0)
    _, rm = _records(orc, dict(base, mirror=0, cloak=0))
    _, rc = _records(orc, dict(base, mirror=1, cloak=1))
    _, rb = _records(orc, dict(base, mirror=1, cloak=0))
    assert np.abs(rm["dir"][:, 2]).max() == 0.0
    # flat-mirror path crossings of the box top y = -A + H on the way in and out
    sc = orc.Scene(base)
    top = base["H"] - base["A"]
    xin = np.zeros(96)
    for i in range(96):
        o, d = orc.camera_dir(sc, i, 0, 0)
        xin[i] = o[0] + (top - o[1]) / d[1] * d[0] if d[1] < 0 else np.inf
    xout = at_plane(rm, top)[:, 0]
    inside = (np.abs(xin) < 19.0) & (np.abs(xout) < 19.0) & (rm["bounces"] == 1)
    assert inside.sum() >= 10
    dd = np.linalg.norm(rc["dir"] - rm["dir"], axis=1)[inside]
    dp = np.linalg.norm(at_plane(rc, top + 1.0) - at_plane(rm, top + 1.0), axis=1)[inside]
    assert dd.max() < 1e-6 and dp.max() < 1e-5, (dd.max(), dp.max())
    assert np.linalg.norm(rb["dir"] - rm["dir"], axis=1)[inside].max() > 0.05


def test_quantize(orc):
    c = np.array([-0.1, 0.0, 0.5 / 255, 0.49 / 255, 1.0, 1.2, 0.5], dtype=np.float32)
    q = orc.quantize(c)
    assert q.tolist() == [0, 0, 1, 0, 255, 255, 128]


def test_texture_bilinear_and_wrap(orc):
    """Texel centres return the texel value; the texture repeats every size
    texels; between centres the value is the bilinear blend of the four
    nearest texels.  Rays are started one unit in front of the background
    plane along its normal, at chosen plane coordinates (s, t)."""
    N, texel = 4, 0.25
    tex = (np.arange(N * N, dtype=np.float32).reshape(N, N) * 7 % 16) / 16.0   # not symmetric
    assert not np.array_equal(tex, tex.T)
    p = inputs.base_scene(width=9, height=9, spp=1, background=1, tex_size=N, tex_texel=texel, mirror=0,
                          cloak=0, azim_deg=25.0)
    sc = orc.Scene(p, tex=tex)
    _, f, r, _, _, _ = _camera_frame(p)
    fr = np.array([f[0], -f[1], f[2]])
    ur = np.cross(r, fr)
    Pb = p["cam_dist"] * fr

    def lookup(s, t):
        rec, _ = orc.trace_from(sc, Pb + s * r + t * ur - fr, fr)
        assert rec["status"] == 0 and rec["bounces"] == 0
        return rec["rgb"]

    for v in range(N):
        for u in range(N):
            s, t = (u + 0.5) * texel, (v + 0.5) * texel
            got = lookup(s, t)
            assert np.abs(got - tex[v, u]).max() < 1e-9, (u, v, got, tex[v, u])
            # one period over in s, in t, and back in both
            for ds, dt in [(N, 0), (0, N), (-N, -N), (3 * N, -2 * N)]:
                assert np.abs(lookup(s + ds * texel, t + dt * texel) - tex[v, u]).max() < 1e-9
    rng = np.random.default_rng(13)
    for s, t in rng.uniform(-3.0, 3.0, size=(40, 2)):
        want = _bilinear_wrap(tex, np.array([s]), np.array([t]), texel)[0]
        assert np.abs(lookup(s, t) - want).max() < 1e-12


def test_texture_background_without_texture_is_an_error(orc):
    p = inputs.base_scene(width=4, height=4, spp=1, background=1, tex_size=8)
    sc = orc.Scene(p)
    with pytest.raises(ValueError):
        orc.render(sc)


# ---------------------------------------------------------------------------
# Closed forms of the background plane and the flat-mirror render, written
# from the scene conventions alone (numpy, no oracle code): the pinhole camera
# of Sec. 4, the mirror reflection at y = 0 and the plane that stands in for
# the photograph of Fig. 2(a).
# ---------------------------------------------------------------------------
def _camera_frame(p):
    """Camera centre C = D (-cos e cos a, sin e, -cos e sin a), view axis
    f = -C / D, right r = f x y / |f x y|, up u = r x f, and the tangents of
    the half fields of view (horizontal from hfov, vertical from the aspect
    ratio, square pixels)."""
    e, a = math.radians(p["elev_deg"]), math.radians(p["azim_deg"])
    D = p["cam_dist"]
    C = D * np.array([-math.cos(e) * math.cos(a), math.sin(e), -math.cos(e) * math.sin(a)])
    f = -C / D
    r = np.cross(f, [0.0, 1.0, 0.0])
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    tx = math.tan(math.radians(p["hfov_deg"]) / 2)
    return C, f, r, u, tx, tx * p["height"] / p["width"]


def _pixel_centre_rays(p):
    """Unit directions through the pixel centres, row-major (H*W, 3)."""
    C, f, r, u, tx, ty = _camera_frame(p)
    H, W = p["height"], p["width"]
    j, i = np.meshgrid(np.arange(W), np.arange(H))
    px = (2.0 * (j + 0.5) / W - 1.0).ravel()
    py = (1.0 - 2.0 * (i + 0.5) / H).ravel()
    d = f[None] + (px * tx)[:, None] * r[None] + (py * ty)[:, None] * u[None]
    return C, d / np.linalg.norm(d, axis=1)[:, None]


def _plane_coords(p, X, d):
    """Where the lines X + t d meet the background plane: normal to the
    mirrored view axis f_r = (f_x, -f_y, f_z), through D f_r, facing the
    origin; returns the coordinates (s, t) along r and u_r = r x f_r and
    whether the line reaches the plane going forward (d . f_r > 0)."""
    _, f, r, _, _, _ = _camera_frame(p)
    fr = np.array([f[0], -f[1], f[2]])
    ur = np.cross(r, fr)
    Pb = p["cam_dist"] * fr
    dn = d @ fr
    with np.errstate(divide="ignore", invalid="ignore"):
        t = ((Pb[None] - X) @ fr) / dn
    Y = X + t[:, None] * d - Pb[None]
    return Y @ r, Y @ ur, dn > 0


def _bilinear_wrap(tex, s, t, texel):
    """Bilinear lookup with texel centres at ((u + 1/2) texel, (v + 1/2) texel),
    rows along t, columns along s, repeating every size texels."""
    N = tex.shape[0]
    U, V = s / texel - 0.5, t / texel - 0.5
    u0, v0 = np.floor(U), np.floor(V)
    fu, fv = U - u0, V - v0
    u0 = u0.astype(np.int64) % N
    v0 = v0.astype(np.int64) % N
    u1, v1 = (u0 + 1) % N, (v0 + 1) % N
    T = tex.astype(np.float64)
    return ((1 - fu) * (1 - fv) * T[v0, u0] + fu * (1 - fv) * T[v0, u1] + (1 - fu) * fv * T[v1, u0]
            + fu * fv * T[v1, u1])


def _flat_mirror_closed_form(p):
    """Exit point, exit direction and whether the background is reached, per
    pixel centre of a flat-mirror scene: the camera ray reflects once at
    y = 0 (d_y -> -d_y) if it descends, then runs straight to the plane."""
    C, d = _pixel_centre_rays(p)
    X = np.repeat(C[None], d.shape[0], 0)
    down = d[:, 1] < 0
    tm = np.where(down, -C[1] / np.where(down, d[:, 1], -1.0), 0.0)
    X[down] = C[None] + tm[down, None] * d[down]
    X[down, 1] = 0.0
    dout = d.copy()
    dout[down, 1] = -d[down, 1]
    return X, dout, down


@pytest.mark.parametrize("elev,azim", [(30.0, 0.0), (10.0, 35.0), (55.0, 80.0)])
def test_flat_mirror_render_closed_form(orc, elev, azim):
    """Every pixel of a flat-mirror checkerboard render equals the closed form:
    exit point and direction within 1e-12, one bounce exactly when the camera
    ray descends, and the colour of cell parity floor(s/cell) + floor(t/cell)
    (colour 0 when even, 0 where the line never reaches the plane)."""
    p = inputs.base_scene(width=48, height=40, spp=1, seed=11, mirror=0, cloak=0, elev_deg=elev, azim_deg=azim)
    X, d, down = _flat_mirror_closed_form(p)
    s, t, ahead = _plane_coords(p, X, d)
    cell = p["bg_cell"]
    parity = (np.floor(s / cell) + np.floor(t / cell)) % 2
    want = np.where((parity == 0)[:, None], np.array(p["colour0"])[None], np.array(p["colour1"])[None])
    want[~ahead] = 0.0
    _, rec = _records(orc, p)
    assert np.abs(rec["pos"] - X).max() < 1e-12
    assert np.abs(rec["dir"] - d).max() < 1e-12
    assert (rec["bounces"] == down.astype(int)).all()
    assert (rec["status"] == np.where(ahead, 0, 1)).all()
    # colours away from cell edges (a line within 1e-9 of an edge may round either way)
    frac_s, frac_t = s / cell - np.floor(s / cell), t / cell - np.floor(t / cell)
    clear = (np.minimum(frac_s, 1 - frac_s) > 1e-9) & (np.minimum(frac_t, 1 - frac_t) > 1e-9)
    assert clear.mean() > 0.99
    assert np.abs(rec["rgb"][clear] - want[clear]).max() < 1e-12
    if elev == 10.0:
        assert (~down).any()              # rays that miss the mirror go straight to the plane
    assert (parity[ahead] == 0).any() and (parity[ahead] == 1).any()


def test_flat_mirror_texture_closed_form(orc):
    """The same render over the bilinear, wrapping texture: every pixel's colour
    within 1e-12 of the closed form."""
    tex = inputs.value_noise(64, seed=12, octaves=3, base_period=16)
    p = inputs.base_scene(width=40, height=36, spp=1, seed=12, mirror=0, cloak=0, background=1, tex_size=64,
                          tex_texel=0.05, azim_deg=20.0)
    X, d, _ = _flat_mirror_closed_form(p)
    s, t, ahead = _plane_coords(p, X, d)
    want = _bilinear_wrap(tex, s, t, p["tex_texel"])
    sc = orc.Scene(p, tex=tex)
    _, rec = orc.render_pixels(sc, np.arange(40 * 36), records=True)
    assert ahead.all()
    assert np.abs(rec["rgb"][:, 0] - want).max() < 1e-12
    assert np.array_equal(rec["rgb"][:, 1], rec["rgb"][:, 0]) and np.array_equal(rec["rgb"][:, 2], rec["rgb"][:, 0])
    # the render covers many texels and wraps the texture at least once
    span = max(np.ptp(s), np.ptp(t)) / p["tex_texel"]
    assert span > 64
