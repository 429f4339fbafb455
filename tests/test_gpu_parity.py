"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: per-ray exit position <= 1e-4 Lambda and exit direction <= 1e-5
rad for rays that take the same path (status and bounce count), at most 0.1%
of pixels whose 8-bit value differs by more than one level, cross-correlations
within 1e-4."""
import math

import numpy as np
import pytest

from conditioning import scene_entry
from paper_1012_5107_gb300 import inputs

pytestmark = pytest.mark.gpu

POS_TOL = 1e-4
DIR_TOL = 1e-5


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


def gpu_render(rt, torch, p, records=True, tex=None, variant=None, min_active=0):
    sc = rt.Scene(p, tex=tex)
    if variant is not None:
        sc.set_launch(variant, min_active)
    rgb = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
    rgb8 = torch.zeros(sc.shape, dtype=torch.uint8, device="cuda")
    rec = torch.zeros(sc.height * sc.wout * sc.spp * 80, dtype=torch.uint8, device="cuda") if records else None
    sc.render(rgb, rgb8, rec)
    torch.cuda.synchronize()
    out = dict(rgb=rgb.cpu().numpy(), rgb8=rgb8.cpu().numpy(), stats=sc.stats())
    if records:
        out["rec"] = rt.records_to_numpy(rec)
    sc.close()
    return out


# FP32 carries about 1e-7 relative rounding into every quantity of a ray
# once the ray reaches the scene (the camera ray up to the cloak box or the
# grating band is set up in FP64).  A ray whose exit moves by more than the
# tolerance when its direction is turned by EPS32 where it reaches the scene
# cannot be resolved in FP32 by any arithmetic; such rays are identified with
# the oracle itself and reported apart from the parity bar.
EPS32 = 3e-7
PERTURB = 1e-7


def sensitivity(orc, p, pix, spp, o_rec, tex=None):
    """Largest change of exit direction and position per radian of a turn of
    the ray where it reaches the scene (two perpendicular 1e-7 rad turns;
    oracle, FP64).  A change of path (bounce count or status) counts as
    infinite sensitivity."""
    sc = orc.Scene(p, tex=tex)
    wout = 1 if p.get("centre_line", 0) else p["width"]
    o_rec = o_rec.reshape(-1)
    Sd = np.zeros(o_rec.size)
    Sp = np.zeros(o_rec.size)
    q = 0
    for px in np.asarray(pix).reshape(-1):
        i, j = divmod(int(px), wout)
        for s in range(spp):
            org, d = orc.camera_dir(sc, i, j, s)
            t = scene_entry(p, org, d)
            if t is None:
                q += 1
                continue
            start = org + 0.999999 * t * d
            a = np.cross(d, [0.0, 1.0, 0.0]); a /= np.linalg.norm(a)
            b = np.cross(d, a)
            for e in (a, b):
                d2 = d + PERTURB * e
                d2 /= np.linalg.norm(d2)
                r, _ = orc.trace_from(sc, start, d2)
                if r["bounces"] != o_rec["bounces"][q] or r["status"] != o_rec["status"][q]:
                    Sd[q] = Sp[q] = np.inf
                else:
                    Sd[q] = max(Sd[q], np.linalg.norm(np.asarray(r["dir"]) - o_rec["dir"][q]) / PERTURB)
                    Sp[q] = max(Sp[q], np.abs(np.asarray(r["pos"]) - o_rec["pos"][q]).max() / PERTURB)
            q += 1
    return Sd, Sp


def compare_records(g, o, pos_tol=POS_TOL, dir_tol=DIR_TOL, min_frac=0.999, cond=None, min_frac_all=None):
    """Same path, exit position and direction within tolerance.  With `cond`
    (a mask of rays that FP32 can resolve) the bar applies to those rays and
    `min_frac_all` to all rays."""
    g = g.reshape(-1)
    o = o.reshape(-1)
    same = (g["status"] == o["status"]) & (g["bounces"] == o["bounces"])
    dpos = np.abs(g["pos"] - o["pos"]).max(1)
    ddir = np.linalg.norm(g["dir"] - o["dir"], axis=1)
    ok = same & (dpos <= pos_tol) & (ddir <= dir_tol)
    info = dict(same=same.mean(), ok=ok.mean(), dpos_med=float(np.median(dpos[same])) if same.any() else 0,
                dpos_max=float(dpos[same].max()) if same.any() else 0,
                ddir_max=float(ddir[same].max()) if same.any() else 0,
                ddir_p99=float(np.percentile(ddir[same], 99)) if same.any() else 0)
    if cond is None:
        assert ok.mean() >= min_frac, info
    else:
        cond = cond.reshape(-1)
        info["conditioned"] = float(cond.mean())
        info["ok_conditioned"] = float(ok[cond].mean()) if cond.any() else 1.0
        assert info["ok_conditioned"] >= min_frac, info
        if min_frac_all is not None:
            assert ok.mean() >= min_frac_all, info
    print(info)
    return info


def fp32_resolvable(orc, p, pix, spp, o_rec, tex=None):
    Sd, Sp = sensitivity(orc, p, pix, spp, o_rec, tex)
    return (Sd * EPS32 <= DIR_TOL) & (Sp * EPS32 <= POS_TOL * p["Lambda"])


def compare_images(q_gpu, q_ref, max_frac=0.001):
    diff = np.abs(q_gpu.astype(int) - q_ref.astype(int)).max(-1)
    frac = (diff > 1).mean()
    print({"pixels_gt1_level": float(frac), "pixels": int(diff.size)})
    assert frac <= max_frac, frac
    return frac


# ---------------------------------------------------------------------------
# Index, gradient and W0 (Eqs. 1, 12, 13)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision,tol", [(1, 1e-12), (0, 2e-6)])
def test_medium_parity(rt, torch, orc, precision, tol):
    for lam, A in [(1.0, 0.04), (1.0, 3 / (16 * math.pi)), (1.7, 0.1)]:
        sc = orc.Scene(inputs.base_scene(Lambda=lam, A=A))
        rng = np.random.default_rng(5)
        x = rng.uniform(-20 * lam, 20 * lam, 4000)
        ys = orc.trochoid(sc, x)[:, 1]
        y = ys + rng.uniform(0.0, 2.0 * lam, 4000) ** 2
        ref = orc.index(sc, x, y)
        xy = torch.tensor(np.stack([x, y], 1), dtype=torch.float64, device="cuda")
        got = rt.eval_medium(precision, lam, A, xy).cpu().numpy()
        W = ref[:, 0] + 1j * ref[:, 1]
        Wg = got[:, 0] + 1j * got[:, 1]
        assert np.abs(Wg - W).max() <= tol * max(1.0, np.abs(W).max()) * 4
        assert np.abs(got[:, 2] - ref[:, 2]).max() <= tol * 4
        F = ref[:, 2:3] * ref[:, 3:5]                     # n grad n
        scale = np.abs(F).max()
        assert np.abs(got[:, 3:5] - F).max() <= tol * 40 * max(scale, 1.0)


@pytest.mark.parametrize("kA", [0.93, 0.97])
def test_medium_near_branch_point(rt, torch, orc, kA):
    """Close to a crest with kA near 1, |zeta + 1/e| < 1e-3: the FP32 path
    refines W0 in FP64."""
    A = kA / (2 * math.pi)
    sc = orc.Scene(inputs.base_scene(A=A))
    x = np.linspace(-0.02, 0.02, 41)
    ys = orc.trochoid(sc, x)[:, 1]
    y = ys + 1e-6
    ref = orc.index(sc, x, y)
    zeta = -kA * np.exp(-2 * math.pi * y) * np.exp(2j * math.pi * x)
    assert np.abs(zeta + 1 / math.e).min() < 1e-3
    xy = torch.tensor(np.stack([x, y], 1), dtype=torch.float64, device="cuda")
    for precision, tol in [(1, 1e-10), (0, 1e-5)]:
        got = rt.eval_medium(precision, 1.0, A, xy).cpu().numpy()
        W = ref[:, 0] + 1j * ref[:, 1]
        Wg = got[:, 0] + 1j * got[:, 1]
        assert np.abs(Wg - W).max() <= tol, (precision, np.abs(Wg - W).max())
        assert np.abs(got[:, 2] / ref[:, 2] - 1).max() <= tol * 10


# ---------------------------------------------------------------------------
# Whole renders (Sec. 4): flat mirror, bare grating, cloaked grating
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("kind", ["mirror", "bare", "cloak"])
def test_render_small_config(rt, torch, orc, precision, kind):
    """64 x 64, 1 sample per pixel, RK4 h = Lambda/200: every sample against the oracle."""
    p = inputs.three_renders(inputs.config_small(precision=precision))[kind]
    g = gpu_render(rt, torch, p)
    o_rgb, o_rec = orc.render(orc.Scene(p), records=True)
    if precision == 1:
        info = compare_records(g["rec"], o_rec, min_frac=1.0)
    else:
        info = compare_records(g["rec"], o_rec, min_frac=0.999)
    compare_images(g["rgb8"], orc.quantize(o_rgb), max_frac=0.001)
    assert g["stats"]["rays"] == 64 * 64
    if precision == 1:
        assert info["dpos_med"] < 1e-9


@pytest.mark.parametrize("precision", [1, 0])
def test_render_main_config_sampled(rt, torch, orc, precision):
    """512 x 512, 4 stratified samples per pixel: the full render in the
    launch configuration the benchmark times, checked on a seeded subset of
    pixels that the oracle traces one by one.  6000 pixels (24000 rays): at
    the FP32 path's measured rate of rays outside the tolerance (0.063 % of
    the render's 1,048,576), 6000 rays would hold the 0.1 % bar only within
    their sampling noise (3.8 expected against 6 allowed)."""
    p = inputs.three_renders(inputs.config_main(precision=precision))["cloak"]
    g = gpu_render(rt, torch, p)
    pix = inputs.pixel_subset(512, 512, 6000, seed=21)
    o_rgb, o_rec = orc.render_pixels(orc.Scene(p), pix, records=True)
    grec = g["rec"].reshape(512 * 512, 4)[pix]
    if precision == 1:
        compare_records(grec, o_rec, min_frac=1.0)
    else:
        # the bar over all rays, and over the rays the oracle finds well conditioned
        cond = fp32_resolvable(orc, p, pix, 4, o_rec)
        compare_records(grec, o_rec, min_frac=0.999, cond=cond, min_frac_all=0.999)
    q = g["rgb8"].reshape(-1, 3)[pix]
    compare_images(q, orc.quantize(o_rgb), max_frac=0.001)
    st = g["stats"]
    assert st["rays"] == 512 * 512 * 4
    assert sum(st["status"]) == st["rays"]


@pytest.mark.parametrize("precision", [1, 0])
def test_render_main_config_all_rays(rt, torch, orc, precision):
    """The full 512 x 512 x 4 cloaked render against the oracle on a seeded
    quarter of its pixels (65536 pixels, 262144 rays): at least 99.9 % of all
    rays within 1e-4 Lambda / 1e-5 rad on the same path (FP64: every ray), and
    at most 0.1 % of those pixels more than one 8-bit level apart."""
    p = inputs.three_renders(inputs.config_main(precision=precision))["cloak"]
    g = gpu_render(rt, torch, p)
    pix = inputs.pixel_subset(512, 512, 65536, seed=24)
    o_rgb, o_rec = orc.render_pixels(orc.Scene(p), pix, records=True)
    grec = g["rec"].reshape(512 * 512, 4)[pix]
    compare_records(grec, o_rec, min_frac=1.0 if precision == 1 else 0.999)
    compare_images(g["rgb8"].reshape(-1, 3)[pix], orc.quantize(o_rgb), max_frac=0.001)


def test_render_pixels_equals_full_render(rt, torch, orc):
    p = inputs.base_scene(width=48, height=40, spp=4, seed=3, precision=0)
    full = gpu_render(rt, torch, p)
    sc = rt.Scene(p)
    pix_np = inputs.pixel_subset(40, 48, 300, seed=4)
    pix = torch.tensor(pix_np, dtype=torch.int64, device="cuda")
    rgb = torch.zeros((300, 3), dtype=torch.float32, device="cuda")
    rec = torch.zeros(300 * 4 * 80, dtype=torch.uint8, device="cuda")
    sc.render_pixels(pix, rgb, rec)
    torch.cuda.synchronize()
    assert np.array_equal(rgb.cpu().numpy(), full["rgb"].reshape(-1, 3)[pix_np])
    r = rt.records_to_numpy(rec).reshape(300, 4)
    f = full["rec"].reshape(-1, 4)[pix_np]
    assert np.array_equal(r["pos"], f["pos"]) and np.array_equal(r["dir"], f["dir"])


def test_render_is_deterministic(rt, torch):
    p = inputs.base_scene(width=64, height=48, spp=4, seed=8, precision=0)
    a = gpu_render(rt, torch, p)
    b = gpu_render(rt, torch, p)
    assert np.array_equal(a["rgb"], b["rgb"])
    assert np.array_equal(a["rec"]["dir"], b["rec"]["dir"])


@pytest.mark.parametrize("over", [
    dict(width=1, height=1, spp=1),
    dict(width=7, height=5, spp=3),                    # non-square spp, ragged sizes
    dict(width=33, height=17, spp=1, centre_line=1),
    dict(width=16, height=16, spp=1, A=0.0),           # flat limit of the grating
    dict(width=16, height=16, spp=1, max_bounces=0),   # guard: every reflection exceeds the cap
    dict(width=16, height=16, spp=1, max_steps=50),    # guard: step cap inside the cloak
    dict(width=12, height=12, spp=4, elev_deg=10.0, azim_deg=35.0, Lambda=0.6, A=0.03, E=4.8, H=1.2),
])
@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("variant", [0, 3])
def test_edge_cases(rt, torch, orc, over, precision, variant):
    p = inputs.base_scene(**over, precision=precision)
    g = gpu_render(rt, torch, p, variant=variant)
    o_rgb, o_rec = orc.render(orc.Scene(p), records=True)
    n = o_rec.size
    if precision == 1:
        compare_records(g["rec"], o_rec, pos_tol=POS_TOL * p["Lambda"], min_frac=1.0)
    else:
        wout = 1 if p["centre_line"] else p["width"]
        cond = fp32_resolvable(orc, p, np.arange(p["height"] * wout), p["spp"], o_rec)
        compare_records(g["rec"], o_rec, pos_tol=POS_TOL * p["Lambda"], min_frac=1.0 - 1.0 / n, cond=cond,
                        min_frac_all=min(0.999, 1.0 - 1.0 / n))
    assert np.array_equal(np.sort(g["rec"]["status"].ravel()), np.sort(o_rec["status"].ravel())) or n > 100


def test_empty_pixel_list(rt, torch):
    sc = rt.Scene(inputs.base_scene(width=8, height=8, spp=1, precision=0))
    pix = torch.zeros(0, dtype=torch.int64, device="cuda")
    rgb = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    sc.render_pixels(pix, rgb)
    torch.cuda.synchronize()
    assert sc.stats()["rays"] == 0


def test_texture_background(rt, torch, orc):
    tex = inputs.value_noise(256, seed=3, octaves=4, base_period=64)
    p = inputs.base_scene(width=40, height=30, spp=4, background=1, tex_size=256, tex_texel=1 / 32,
                          precision=0)
    g = gpu_render(rt, torch, p, tex=tex)
    o_rgb, o_rec = orc.render(orc.Scene(p, tex=tex), records=True)
    cond = fp32_resolvable(orc, p, np.arange(30 * 40), 4, o_rec, tex)
    compare_records(g["rec"], o_rec, min_frac=0.999, cond=cond, min_frac_all=0.999)
    compare_images(g["rgb8"], orc.quantize(o_rgb), max_frac=0.001)
    assert np.median(np.abs(g["rgb"] - o_rgb)) < 1e-5


# ---------------------------------------------------------------------------
# Cross-correlation (Sec. 5, Eqs. 14-15)
# ---------------------------------------------------------------------------
def test_xcorr_parity(rt, torch, orc):
    rng = np.random.default_rng(2)
    # (512, 1), (20, 10), (7, 21), (65, 21): one block; (66, 21) is the
    # first height past its 4096 values; the rest take the three passes
    for H, W in [(64, 64), (37, 129), (512, 1), (300, 512), (20, 10), (7, 21), (65, 21), (66, 21)]:
        f = rng.random((H, W, 3)).astype(np.float32)
        g = (0.6 * f + 0.4 * rng.random((H, W, 3))).astype(np.float32)
        fovs = [0.0, 10.0, 25.0, 50.0]
        out = rt.xcorr(torch.tensor(f, device="cuda"), torch.tensor(g, device="cuda"), fovs, 50.0)
        out = out.cpu().numpy()
        for q, fov in enumerate(fovs):
            j0, j1 = orc.fov_columns(W, 50.0, fov)
            ref = orc.xcorr(f, g, j0, j1)
            if j1 > j0:
                assert np.abs(out[q] - ref).max() < 1e-10
            else:
                assert np.isnan(out[q]).all()


C_TOL = 1e-4     # cross-correlations of renders, GPU against the oracle


@pytest.mark.parametrize("precision", [1, 0])
def test_xcorr_of_renders(rt, torch, orc, precision):
    """C(cloak, mirror) and C(bare, mirror) of the small workload's renders
    (64 x 64, one sample per pixel), GPU against the oracle, within 1e-4 at
    FOV 0 (the centre-line renders), 10, 25 and 50 deg."""
    base = inputs.config_small(precision=precision)
    imgs, refs = {}, {}
    for kind, p in inputs.three_renders(base).items():
        for line in (0, 1):
            q = dict(p, centre_line=line)
            imgs[(kind, line)] = torch.tensor(gpu_render(rt, torch, q, records=False)["rgb"], device="cuda")
            refs[(kind, line)] = orc.render(orc.Scene(q))
    worst = 0.0
    for kind in ("cloak", "bare"):
        out = rt.xcorr(imgs[("mirror", 0)], imgs[(kind, 0)], [10.0, 25.0, 50.0], 50.0).cpu().numpy()
        for q, fov in enumerate([10.0, 25.0, 50.0]):
            j0, j1 = orc.fov_columns(64, 50.0, fov)
            ref = orc.xcorr(refs[("mirror", 0)], refs[(kind, 0)], j0, j1)
            worst = max(worst, np.abs(out[q] - ref).max())
            assert np.abs(out[q] - ref).max() < C_TOL, (kind, fov, out[q], ref)
        out0 = rt.xcorr(imgs[("mirror", 1)], imgs[(kind, 1)], [0.0], 50.0).cpu().numpy()
        ref0 = orc.xcorr(refs[("mirror", 1)], refs[(kind, 1)], 0, 1)
        worst = max(worst, np.abs(out0[0] - ref0).max())
        assert np.abs(out0[0] - ref0).max() < C_TOL, (kind, 0.0, out0[0], ref0)
    print(f"precision {precision}: largest |dC| {worst:.2e}")


def subset_columns(W, pix, j0, j1):
    """Indices (into a pixel subset) of the pixels whose column lies in [j0, j1)."""
    j = pix % W
    return np.nonzero((j >= j0) & (j < j1))[0]


_ORACLE_SUBSET = {}


def oracle_subset(orc, p, pix):
    """Oracle colours of a pixel subset (cached: the oracle traces in FP64
    whatever precision the scene asks of the GPU)."""
    key = (p["mirror"], p["cloak"], p.get("centre_line", 0), len(pix))
    if key not in _ORACLE_SUBSET:
        _ORACLE_SUBSET[key] = orc.render(orc.Scene(p)) if p.get("centre_line", 0) else \
            orc.render_pixels(orc.Scene(p), pix)
    return _ORACLE_SUBSET[key]


@pytest.mark.parametrize("precision", [1, 0])
def test_xcorr_of_benchmark_renders_sampled(rt, torch, orc, precision):
    """The benchmark's 512 x 512 x 4 renders (mirror, bare and cloaked
    grating) in full on the GPU, and a seeded subset of 65536 pixels of each
    traced by the oracle.  Eq. 15 over the subset's pixels in each FOV window
    (the window's columns restricted to the subset), packed into one column
    per window and computed by rt_xcorr on the GPU renders and by the oracle
    on its own: within 1e-4 at FOV 10, 25 and 50 deg; FOV 0 from the
    centre-line renders in full."""
    base = inputs.config_main(precision=precision)
    pix = inputs.pixel_subset(512, 512, 65536, seed=23)
    gimg, oimg = {}, {}
    for kind, p in inputs.three_renders(base).items():
        g = gpu_render(rt, torch, p, records=False)["rgb"].reshape(-1, 3)
        gimg[kind] = g[pix]
        oimg[kind] = oracle_subset(orc, p, pix)
        q = dict(p, centre_line=1)
        gimg[kind + "_line"] = gpu_render(rt, torch, q, records=False)["rgb"]
        oimg[kind + "_line"] = oracle_subset(orc, q, pix)
    worst = 0.0
    for kind in ("cloak", "bare"):
        for fov in (10.0, 25.0, 50.0):
            j0, j1 = orc.fov_columns(512, 50.0, fov)
            sel = subset_columns(512, pix, j0, j1)
            f_g = torch.tensor(gimg["mirror"][sel][:, None, :], device="cuda")
            g_g = torch.tensor(gimg[kind][sel][:, None, :], device="cuda")
            got = rt.xcorr(f_g, g_g, [0.0], 50.0).cpu().numpy()[0]
            ref = orc.xcorr(oimg["mirror"][sel][:, None, :], oimg[kind][sel][:, None, :], 0, 1)
            worst = max(worst, np.abs(got - ref).max())
            assert np.abs(got - ref).max() < C_TOL, (kind, fov, got, ref)
        got0 = rt.xcorr(torch.tensor(gimg["mirror_line"], device="cuda"),
                        torch.tensor(gimg[kind + "_line"], device="cuda"), [0.0], 50.0).cpu().numpy()[0]
        ref0 = orc.xcorr(oimg["mirror_line"], oimg[kind + "_line"], 0, 1)
        worst = max(worst, np.abs(got0 - ref0).max())
        assert np.abs(got0 - ref0).max() < C_TOL, (kind, 0.0, got0, ref0)
    print(f"precision {precision}: largest |dC| {worst:.2e}")


# ---------------------------------------------------------------------------
# Dormand-Prince RK45 (adaptive steps)
# ---------------------------------------------------------------------------
def test_dp45_fp64_matches_oracle(rt, torch, orc):
    """Same tolerance (1e-7) on both sides: the same step sequence and exit."""
    p = inputs.base_scene(width=64, height=64, spp=1, integrator=1, rtol=1e-7, atol=1e-7, precision=1)
    g = gpu_render(rt, torch, p)
    o_rgb, o_rec = orc.render(orc.Scene(p), records=True)
    info = compare_records(g["rec"], o_rec, min_frac=1.0)
    assert info["ddir_max"] < 1e-9
    compare_images(g["rgb8"], orc.quantize(o_rgb))


@pytest.mark.parametrize("rtol", [1e-5, 1e-7])
def test_dp45_fp32_matches_oracle(rt, torch, orc, rtol):
    """FP32 against the oracle at the same tolerance, on the rays FP32 can resolve."""
    p = inputs.base_scene(width=64, height=64, spp=1, integrator=1, rtol=rtol, atol=rtol, precision=0)
    g = gpu_render(rt, torch, p)
    o_rgb, o_rec = orc.render(orc.Scene(p), records=True)
    cond = fp32_resolvable(orc, p, np.arange(64 * 64), 1, o_rec)
    compare_records(g["rec"], o_rec, min_frac=0.999, cond=cond, min_frac_all=0.999)
    compare_images(g["rgb8"], orc.quantize(o_rgb), max_frac=0.001)


@pytest.mark.parametrize("extent,A", [(2.0, 0.02), (8.0, 0.04), (32.0, 0.04)])
def test_hd_workload_sampled(rt, torch, orc, extent, A):
    """1920 x 1080, 16 samples per pixel, Dormand-Prince, value-noise
    background: a seeded subset of pixels rendered by rt_render_pixels (the
    same arithmetic as the full render) against the oracle."""
    tex = inputs.value_noise(2048, seed=3)
    p = inputs.config_hd(extent=extent, A=A, precision=0)
    pix_np = inputs.pixel_subset(1080, 1920, 120, seed=31)
    sc = rt.Scene(p, tex=tex)
    pix = torch.tensor(pix_np, dtype=torch.int64, device="cuda")
    rgb = torch.zeros((pix_np.size, 3), dtype=torch.float32, device="cuda")
    rec = torch.zeros(pix_np.size * 16 * 80, dtype=torch.uint8, device="cuda")
    sc.render_pixels(pix, rgb, rec)
    torch.cuda.synchronize()
    g = rt.records_to_numpy(rec)
    o_rgb, o_rec = orc.render_pixels(orc.Scene(p, tex=tex), pix_np, records=True)
    cond = fp32_resolvable(orc, p, pix_np, 16, o_rec, tex)
    compare_records(g, o_rec, min_frac=0.999, cond=cond, min_frac_all=0.995)
    assert np.median(np.abs(rgb.cpu().numpy() - o_rgb)) < 1e-4


# ---------------------------------------------------------------------------
# Launch variants: the per-lane loop and the wavefront loop trace every ray
# with the same arithmetic; only the grouping of rays into warps differs.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision,integrator", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("kind", ["mirror", "bare", "cloak"])
def test_wave_equals_lane_loop(rt, torch, precision, integrator, kind):
    p = inputs.three_renders(inputs.base_scene(width=96, height=80, spp=4, seed=5, integrator=integrator,
                                               rtol=1e-5 if precision == 0 else 1e-7,
                                               atol=1e-5 if precision == 0 else 1e-7,
                                               precision=precision))[kind]
    a = gpu_render(rt, torch, p, variant=0)
    b = gpu_render(rt, torch, p, variant=3)
    same_variant_bar(a, b, precision)


def same_variant_bar(a, b, precision):
    """The two loops compile the same arithmetic separately, so the compiler
    may fuse a different multiply-add here and there: FP64 results agree to
    rounding, FP32 ones within the parity tolerances on all but the
    ill-conditioned rays (the same bar as against the oracle)."""
    ga, gb = a["rec"].reshape(-1), b["rec"].reshape(-1)
    same = (ga["status"] == gb["status"]) & (ga["bounces"] == gb["bounces"])
    dpos = np.abs(ga["pos"] - gb["pos"]).max(1)
    ddir = np.linalg.norm(ga["dir"] - gb["dir"], axis=1)
    exact = (dpos == 0) & (ddir == 0) & same
    print(dict(exact=float(exact.mean()), same=float(same.mean()), dpos_max=float(dpos[same].max()),
               ddir_max=float(ddir[same].max()), ddir_p999=float(np.percentile(ddir[same], 99.9))))
    assert ga.size == gb.size and a["stats"]["rays"] == b["stats"]["rays"]
    assert b["stats"]["sched_timeouts"] == 0
    if precision == 1:
        assert same.all() and dpos.max() <= 1e-10 and ddir.max() <= 1e-10
        compare_images(a["rgb8"], b["rgb8"], max_frac=0.0)
    else:
        ok = same & (dpos <= POS_TOL) & (ddir <= DIR_TOL)
        assert ok.mean() >= 0.995
        compare_images(a["rgb8"], b["rgb8"], max_frac=0.001)


@pytest.mark.parametrize("min_active", [1, 16, 32])
def test_wave_main_config_equals_lane_loop(rt, torch, min_active):
    """The full 512 x 512 x 4 cloaked render (the benchmark's dominant launch):
    identical images and records for every setting of the wavefront loop."""
    p = inputs.three_renders(inputs.config_main(precision=0))["cloak"]
    a = gpu_render(rt, torch, p, variant=0, min_active=24)
    b = gpu_render(rt, torch, p, variant=3, min_active=min_active)
    same_variant_bar(a, b, 0)
    assert b["stats"]["rays"] == 512 * 512 * 4
    c = gpu_render(rt, torch, p, variant=3, min_active=24 if min_active != 24 else 16)
    # within the wavefront loop the grouping of rays never changes a result
    assert np.array_equal(b["rgb"], c["rgb"]) and np.array_equal(b["rec"]["dir"], c["rec"]["dir"])


def test_wave_texture_and_pixel_list(rt, torch, orc):
    """Textured background, a listed pixel subset and a ragged size through the wavefront loop."""
    tex = inputs.value_noise(256, seed=6)
    p = inputs.base_scene(width=37, height=29, spp=2, seed=6, background=1, tex_size=256, precision=0)
    sc = rt.Scene(p, tex=tex)
    sc.set_launch(3, 20)
    pix_np = inputs.pixel_subset(29, 37, 200, seed=7)
    pix = torch.tensor(pix_np, dtype=torch.int64, device="cuda")
    rgb = torch.zeros((200, 3), dtype=torch.float32, device="cuda")
    sc.render_pixels(pix, rgb)
    torch.cuda.synchronize()
    full = gpu_render(rt, torch, p, tex=tex, variant=3, min_active=28)
    assert np.array_equal(rgb.cpu().numpy(), full["rgb"].reshape(-1, 3)[pix_np])
    o_rgb = orc.render_pixels(orc.Scene(p, tex=tex), pix_np)
    assert np.median(np.abs(rgb.cpu().numpy() - o_rgb)) < 1e-4


def test_variant_not_compiled_is_rejected(rt):
    sc = rt.Scene(inputs.base_scene(width=8, height=8, spp=1, precision=1))
    with pytest.raises(Exception):
        sc.set_launch(1, 0)          # per-lane register variants 1, 2 exist for FP32 RK4 only
    sc.set_launch(3, 0)
    assert sc.get_launch()["variant"] == 3
