"""The time form of Eq. 11 (integrator RT_RK4T: classical RK4 on (r, v) in
physical time t, |v| = c0/n) on the GPU against the oracle's integrator 2:
every sample of small renders in FP64, the rays FP32 can resolve, the
velocity-momentum conversions at the faces (Fresnel branches, the referenced
cloak), the batch, and the launch variants it does not have."""
import numpy as np
import pytest

from paper_1012_5107_gb300 import inputs
from test_gpu_parity import compare_images, compare_records, fp32_resolvable, gpu_render, same_variant_bar

pytestmark = pytest.mark.gpu

RK4T = 2


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


@pytest.mark.parametrize("over", [
    dict(),
    dict(width=33, height=17, spp=3, seed=2),                                     # ragged, non-square spp
    dict(elev_deg=10.0, azim_deg=35.0, Lambda=0.6, A=0.03, E=4.8, H=1.2),          # 3-D rays, v_z varies
    dict(max_steps=50),                                                           # step guard in the box
    dict(h=1.0 / 80),                                                             # coarse step
])
def test_fp64_matches_oracle(rt, torch, orc, over):
    q = dict(width=64, height=64, spp=1, seed=13, integrator=RK4T, precision=1)
    q.update(over)
    p = inputs.base_scene(**q)
    g = gpu_render(rt, torch, p)
    o_rgb, o_rec = orc.render(orc.Scene(p), records=True)
    info = compare_records(g["rec"], o_rec, pos_tol=1e-4 * p["Lambda"], min_frac=1.0)
    assert info["dpos_med"] < 1e-9 and info["ddir_max"] < 1e-7
    compare_images(g["rgb8"], orc.quantize(o_rgb))
    assert g["stats"]["sched_timeouts"] == 0


def test_fp32_matches_oracle(rt, torch, orc):
    p = inputs.base_scene(width=64, height=64, spp=1, seed=14, integrator=RK4T, precision=0)
    g = gpu_render(rt, torch, p)
    o_rgb, o_rec = orc.render(orc.Scene(p), records=True)
    cond = fp32_resolvable(orc, p, np.arange(64 * 64), 1, o_rec)
    compare_records(g["rec"], o_rec, min_frac=0.999, cond=cond, min_frac_all=0.998)
    compare_images(g["rgb8"], orc.quantize(o_rgb), max_frac=0.001)


def test_main_config_sampled(rt, torch, orc):
    """512 x 512 x 4 cloaked render in FP32 with the time form: a seeded
    subset of pixels against the oracle."""
    p = inputs.three_renders(dict(inputs.config_main(precision=0), integrator=RK4T))["cloak"]
    g = gpu_render(rt, torch, p)
    pix = inputs.pixel_subset(512, 512, 600, seed=22)
    o_rgb, o_rec = orc.render_pixels(orc.Scene(p), pix, records=True)
    grec = g["rec"].reshape(512 * 512, 4)[pix]
    cond = fp32_resolvable(orc, p, pix, 4, o_rec)
    compare_records(grec, o_rec, min_frac=0.999, cond=cond, min_frac_all=0.998)
    compare_images(g["rgb8"].reshape(-1, 3)[pix], orc.quantize(o_rgb), max_frac=0.001)
    assert g["stats"]["rays"] == 512 * 512 * 4


@pytest.mark.parametrize("flags", [1, 4, 5])
def test_fp64_options_match_oracle(rt, torch, orc, flags):
    """Referenced cloak (flag 1), Fresnel weights (4) and both: the velocity is
    turned into the momentum at every face and back at a branch's start."""
    p = inputs.base_scene(width=48, height=40, spp=2, seed=15, integrator=RK4T, precision=1, flags=flags)
    g = gpu_render(rt, torch, p)
    o_rgb, o_rec = orc.render(orc.Scene(p), records=True)
    gr, orr = g["rec"].reshape(-1), o_rec.reshape(-1)
    same = (gr["status"] == orr["status"]) & (gr["bounces"] == orr["bounces"])
    assert same.mean() >= 0.999
    assert np.abs(gr["pos"] - orr["pos"])[same].max() < 1e-9
    assert np.abs(gr["dir"] - orr["dir"])[same].max() < 1e-9
    assert (np.abs(g["rgb"] - o_rgb).max(-1) > 1e-6).mean() <= 0.002


def test_time_form_traces_the_tau_form_curves(rt, torch):
    """Both forms integrate the same rays (Eq. 11 and its Hamiltonian form
    differ by the parametrisation dtau = c0/n^2 dt): at a fine step their
    exits agree to the integrators' truncation error."""
    base = inputs.base_scene(width=48, height=48, spp=1, seed=16, h=1.0 / 800, precision=1)
    a = gpu_render(rt, torch, base)
    b = gpu_render(rt, torch, dict(base, integrator=RK4T))
    ga, gb = a["rec"].reshape(-1), b["rec"].reshape(-1)
    same = (ga["status"] == gb["status"]) & (ga["bounces"] == gb["bounces"])
    assert same.mean() >= 0.995
    assert np.abs(ga["pos"] - gb["pos"])[same].max() < 1e-6
    assert np.linalg.norm(ga["dir"] - gb["dir"], axis=1)[same].max() < 1e-6


def test_batch_equals_single_renders(rt, torch):
    ps = [inputs.base_scene(width=40, height=32, spp=2, seed=17 + q, scene_id=q, integrator=RK4T, precision=0)
          for q in range(3)]
    scenes = [rt.Scene(p) for p in ps]
    outs = [torch.zeros(s.shape, dtype=torch.float32, device="cuda") for s in scenes]
    b = rt.Batch(scenes)
    b.render(outs)
    torch.cuda.synchronize()
    for p, o in zip(ps, outs):
        single = gpu_render(rt, torch, p, records=False)
        assert np.array_equal(o.cpu().numpy(), single["rgb"])
    assert b.stats()["sched_timeouts"] == 0
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_grouping_does_not_change_results(rt, torch, precision):
    p = inputs.base_scene(width=64, height=48, spp=4, seed=18, integrator=RK4T, precision=precision)
    a = gpu_render(rt, torch, p, variant=3, min_active=28)
    b = gpu_render(rt, torch, p, variant=3, min_active=1)
    same_variant_bar(a, b, precision)
    assert np.array_equal(a["rgb"], b["rgb"])


def test_only_the_wavefront_loop(rt):
    sc = rt.Scene(inputs.base_scene(width=8, height=8, spp=1, integrator=RK4T, precision=0))
    for v in (0, 1, 2):
        with pytest.raises(rt.RtError):
            sc.set_launch(v, 0)
    sc.set_launch(3, 20)
    assert sc.get_launch()["variant"] == 3
    sc.close()
