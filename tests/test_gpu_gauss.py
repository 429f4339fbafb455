"""The Gaussian conformal cloak (Sec. 2, Fig. 1(b), Fig. 4; the bump of
Eq. 5 in its exact form) on the GPU against the oracle: every sample of small
renders of the bare and the cloaked bump in FP64, the rays FP32 can resolve,
Dormand-Prince, edge cases, C(0,0) of the Fig. 4 pairs, a sampled full-size
render, and the calls that do not take Gaussian scenes."""
import numpy as np
import pytest

from paper_1012_5107_gb300 import inputs
from test_gpu_parity import DIR_TOL, POS_TOL, compare_images, compare_records, fp32_resolvable, gpu_render

pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def scene_entry(p, org, d):
    """Where the camera ray reaches the Gaussian scene: the band y <= h or the
    cloak box (y from 0 to H)."""
    ts = []
    if d[1] < 0.0:
        ts.append((max(p["A"], 1e-6) - org[1]) / d[1])
    if p["cloak"]:
        lo = np.array([-p["E"] / 2, 0.0, -p["E"] / 2])
        hi = np.array([p["E"] / 2, p["H"], p["E"] / 2])
        with np.errstate(divide="ignore", invalid="ignore"):
            t1, t2 = (lo - org) / d, (hi - org) / d
        tn, tf = np.minimum(t1, t2).max(), np.maximum(t1, t2).min()
        if tn <= tf and tn > 0:
            ts.append(tn)
    ts = [t for t in ts if t > 0]
    return min(ts) if ts else None


@pytest.fixture(autouse=True)
def _gauss_entry(monkeypatch):
    # the FP32 sensitivity probe starts the perturbed rays where they reach the scene
    import test_gpu_parity
    monkeypatch.setattr(test_gpu_parity, "scene_entry", scene_entry)


@pytest.mark.parametrize("kind", ["bare", "cloak"])
@pytest.mark.parametrize("precision", [1, 0])
def test_small_renders_match_oracle(rt, torch, orc, kind, precision):
    """64 x 64, one sample per pixel, RK4 h = Lambda/200 (Fig. 4 b, c)."""
    p = inputs.gauss_renders(inputs.gauss_scene(width=64, height=64, spp=1, seed=1, precision=precision))[kind]
    g = gpu_render(rt, torch, p)
    o_rgb, o_rec = orc.render(orc.Scene(p), records=True)
    if precision == 1:
        info = compare_records(g["rec"], o_rec, min_frac=1.0)
        assert info["dpos_med"] < 1e-9 and info["ddir_max"] < 1e-8
        compare_images(g["rgb8"], orc.quantize(o_rgb))
    else:
        cond = fp32_resolvable(orc, p, np.arange(64 * 64), 1, o_rec)
        compare_records(g["rec"], o_rec, min_frac=0.999, cond=cond, min_frac_all=0.998)
        compare_images(g["rgb8"], orc.quantize(o_rgb), max_frac=0.001)
    assert g["stats"]["rays"] == 64 * 64 and g["stats"]["sched_timeouts"] == 0


@pytest.mark.parametrize("precision,rtol", [(1, 1e-7), (0, 1e-5)])
def test_dp45_matches_oracle(rt, torch, orc, precision, rtol):
    p = inputs.gauss_scene(width=48, height=48, spp=1, seed=2, integrator=1, rtol=rtol, atol=rtol,
                           precision=precision)
    g = gpu_render(rt, torch, p)
    o_rgb, o_rec = orc.render(orc.Scene(p), records=True)
    if precision == 1:
        info = compare_records(g["rec"], o_rec, min_frac=1.0)
        assert info["ddir_max"] < 1e-8
    else:
        cond = fp32_resolvable(orc, p, np.arange(48 * 48), 1, o_rec)
        compare_records(g["rec"], o_rec, min_frac=0.999, cond=cond, min_frac_all=0.998)
    compare_images(g["rgb8"], orc.quantize(o_rgb), max_frac=0.001)


@pytest.mark.parametrize("over", [
    dict(width=1, height=1, spp=1),
    dict(width=7, height=5, spp=3),                                   # ragged, non-square spp
    dict(width=33, height=17, spp=1, centre_line=1),                  # the 2-D line of Table 1
    dict(width=16, height=16, spp=1, A=0.0),                          # flat limit: n = 1 in the box
    dict(width=16, height=16, spp=1, max_bounces=0),
    dict(width=16, height=16, spp=1, max_steps=50),
    dict(width=12, height=12, spp=4, elev_deg=10.0, azim_deg=35.0, gauss_w=0.5, A=0.3, E=3.0, H=1.5),
])
def test_edge_cases_fp64(rt, torch, orc, over):
    p = inputs.gauss_scene(precision=1, **over)
    g = gpu_render(rt, torch, p)
    o_rgb, o_rec = orc.render(orc.Scene(p), records=True)
    compare_records(g["rec"], o_rec, pos_tol=POS_TOL * p["Lambda"], min_frac=1.0)
    assert np.array_equal(np.sort(g["rec"]["status"].ravel()), np.sort(o_rec["status"].ravel()))


def test_fig4_correlations_match_oracle(rt, torch, orc):
    """C(0,0) of Fig. 4(a) against 4(b) and 4(c) at FOV 0/10/25/50 deg (the
    Gaussian rows of Table 1) on FP64 renders, GPU against oracle."""
    base = inputs.gauss_scene(width=96, height=80, spp=1, seed=4, precision=1)
    r = inputs.gauss_renders(base)
    line = {k: dict(v, centre_line=1) for k, v in r.items()}
    g, o = {}, {}
    for name, p in list(r.items()) + [("line_" + k, v) for k, v in line.items()]:
        g[name] = torch.from_numpy(gpu_render(rt, torch, p, records=False)["rgb"]).cuda()
        o[name] = orc.render(orc.Scene(p))
    for other in ("bare", "cloak"):
        cg = rt.xcorr(g["mirror"], g[other], [10.0, 25.0, 50.0], 50.0).cpu().numpy()
        co = np.array([orc.xcorr(o["mirror"], o[other], *orc.fov_columns(96, 50.0, f)) for f in (10.0, 25.0, 50.0)])
        assert np.abs(cg - co).max() < 1e-4
        lg = rt.xcorr(g["line_mirror"], g["line_" + other], [50.0], 50.0).cpu().numpy()
        lo = orc.xcorr(o["line_mirror"], o["line_" + other], 0, 1)
        assert np.abs(lg[0] - lo).max() < 1e-4


def test_main_size_sampled(rt, torch, orc):
    """512 x 512 x 4 cloaked bump, FP32, against the oracle on a seeded subset."""
    p = inputs.gauss_scene(width=512, height=512, spp=4, seed=2, precision=0)
    g = gpu_render(rt, torch, p)
    pix = inputs.pixel_subset(512, 512, 500, seed=23)
    o_rgb, o_rec = orc.render_pixels(orc.Scene(p), pix, records=True)
    grec = g["rec"].reshape(512 * 512, 4)[pix]
    cond = fp32_resolvable(orc, p, pix, 4, o_rec)
    compare_records(grec, o_rec, min_frac=0.999, cond=cond, min_frac_all=0.998)
    compare_images(g["rgb8"].reshape(-1, 3)[pix], orc.quantize(o_rgb), max_frac=0.001)
    st = g["stats"]
    assert st["rays"] == 512 * 512 * 4 and sum(st["status"]) == st["rays"] and st["sched_timeouts"] == 0


def test_grouping_does_not_change_results(rt, torch):
    p = inputs.gauss_scene(width=64, height=48, spp=4, seed=5, precision=0)
    a = gpu_render(rt, torch, p, variant=3, min_active=28)
    b = gpu_render(rt, torch, p, variant=3, min_active=1)
    assert np.array_equal(a["rgb"], b["rgb"]) and np.array_equal(a["rec"]["dir"], b["rec"]["dir"])


def test_calls_that_do_not_take_gaussian_scenes(rt, torch):
    p = inputs.gauss_scene(width=8, height=8, spp=1, precision=0)
    sc = rt.Scene(p)
    for v in (0, 1, 2):
        with pytest.raises(rt.RtError):
            sc.set_launch(v, 0)
    with pytest.raises(rt.RtError):
        rt.Batch([sc])
    sc.close()


@pytest.mark.parametrize("bad,msg", [
    (dict(gauss_w=0.0), "gauss_w"), (dict(A=0.3), "0.8 gauss_w"), (dict(flags=4), "no options"),
    (dict(integrator=2), "RT_RK4 or RT_DP45"), (dict(H=0.1), "H > A"),
])
def test_invalid_gaussian_scenes(rt, bad, msg):
    with pytest.raises(rt.RtError) as e:
        rt.Scene(inputs.gauss_scene(**bad))
    assert msg in str(e.value)
