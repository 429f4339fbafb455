"""Pins for the oracle's camera, sampling, backgrounds and whole renders (Sec. 4)."""
import json
import math
import os

import numpy as np

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
    """Texel centres return the texel value; the texture repeats every size texels."""
    tex = np.arange(16, dtype=np.float32).reshape(4, 4) / 16.0
    p = inputs.base_scene(width=9, height=9, spp=1, background=1, tex_texel=0.25, mirror=0, cloak=0)
    sc = orc.Scene(p, tex=tex)
    rgb, rec = orc.render_pixels(sc, np.arange(81), records=True)
    assert np.all((rgb >= 0) & (rgb <= 15 / 16 + 1e-6))
    assert np.allclose(rgb[:, 0], rgb[:, 1]) and np.allclose(rgb[:, 0], rgb[:, 2])


def test_texture_background_without_texture_is_an_error(orc):
    import pytest
    p = inputs.base_scene(width=4, height=4, spp=1, background=1, tex_size=8)
    sc = orc.Scene(p)
    with pytest.raises(ValueError):
        orc.render(sc)
