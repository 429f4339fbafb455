"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds none of the method's arithmetic: it only produces scene
parameter dictionaries (geometry, camera, integrator settings), the
checkerboard colours, the value-noise texture that stands in for the paper's
input photograph (Sec. 4, Fig. 2a) and seeded pixel subsets.  It imports only
numpy, so importing it never loads the CUDA library.

All lengths are world units; the grating period Lambda sets the scale.
"""
from __future__ import annotations

import math

import numpy as np

RK4, DP45 = 0, 1
FP32, FP64 = 0, 1
FLAT, TROCHOID, GAUSS = 0, 1, 2
CHECKER, TEXTURE = 0, 1


def checker_colours(seed: int) -> tuple[tuple[float, ...], tuple[float, ...]]:
    """Two 8-bit RGB colours drawn from the seed, as floats in [0, 1]."""
    rng = np.random.default_rng([seed, 0xC0105])
    c = rng.integers(0, 256, size=(2, 3))
    # keep the two colours distinguishable in every channel
    c[1] = (c[0] + 64 + rng.integers(0, 128, size=3)) % 256
    return tuple(float(v) / 255.0 for v in c[0]), tuple(float(v) / 255.0 for v in c[1])


def value_noise(size: int = 2048, seed: int = 3, octaves: int = 4, base_period: int = 256) -> np.ndarray:
    """Seeded periodic value noise (size x size float32 in [0, 1]): random lattice
    values per octave, smoothstep-interpolated, octaves halving in period and
    amplitude.  The texture wraps seamlessly because every period divides size."""
    rng = np.random.default_rng([seed, 0x7E47])
    out = np.zeros((size, size), dtype=np.float64)
    amp, total = 1.0, 0.0
    period = base_period
    idx = np.arange(size)
    for _ in range(octaves):
        n = size // period
        lat = rng.random((n, n))
        u = (idx % period) / period
        u = u * u * (3.0 - 2.0 * u)
        i0 = idx // period
        i1 = (i0 + 1) % n
        a = lat[i0][:, i0]
        b = lat[i0][:, i1]
        c = lat[i1][:, i0]
        d = lat[i1][:, i1]
        uu = u[None, :]
        vv = u[:, None]
        out += amp * ((1 - vv) * ((1 - uu) * a + uu * b) + vv * ((1 - uu) * c + uu * d))
        total += amp
        amp *= 0.5
        period //= 2
    out /= total
    lo, hi = out.min(), out.max()
    return ((out - lo) / (hi - lo)).astype(np.float32)


def base_scene(**over) -> dict:
    """The 64x64 single-sample RK4 workload: Lambda = 1, A = 0.04 (kA ~ 0.25),
    cloak box 2 Lambda high above y = -A and 8 Lambda wide in x and z, pinhole
    camera 12 Lambda away at 30 degrees elevation with a 50 degree horizontal
    field of view, seeded checkerboard background with 0.5 Lambda cells."""
    c0, c1 = checker_colours(over.get("seed", 1))
    p = dict(
        Lambda=1.0, A=0.04, H=2.0, E=8.0,
        cam_dist=12.0, elev_deg=30.0, azim_deg=0.0, hfov_deg=50.0,
        bg_cell=0.5, tex_texel=1.0 / 32.0, colour0=c0, colour1=c1,
        h=1.0 / 200.0, rtol=1e-7, atol=1e-7, h_max=1.0 / 16.0, gauss_w=0.306,
        seed=1, scene_id=0, max_steps=1 << 20,
        mirror=TROCHOID, cloak=1, width=64, height=64, spp=1, centre_line=0,
        background=CHECKER, tex_size=0, integrator=RK4, max_bounces=16,
        precision=FP64,
    )
    p.update(over)
    if "seed" in over and "colour0" not in over:
        p["colour0"], p["colour1"] = checker_colours(over["seed"])
    # lengths that scale with Lambda when only Lambda was overridden
    return p


def scale_scene(p: dict, lam: float) -> dict:
    """The same scene with every length multiplied by lam (renders are invariant)."""
    q = dict(p)
    for key in ("Lambda", "A", "H", "E", "cam_dist", "bg_cell", "tex_texel", "h", "h_max", "atol", "gauss_w"):
        q[key] = p[key] * lam
    return q


def three_renders(p: dict) -> dict[str, dict]:
    """Flat mirror, bare grating and cloaked grating versions of one scene
    (Fig. 3 a, b, c)."""
    return {
        "mirror": dict(p, mirror=FLAT, cloak=0),
        "bare": dict(p, mirror=TROCHOID, cloak=0),
        "cloak": dict(p, mirror=TROCHOID, cloak=1),
    }


def gauss_scene(**over) -> dict:
    """The Gaussian conformal cloak of Fig. 1(b) and Fig. 4: bump width
    w = 0.306 and height h = 0.13 (A holds h), cloak box 1.1 high above the
    flat mirror and 8 wide, otherwise the base scene."""
    q = dict(mirror=GAUSS, A=0.13, gauss_w=0.306, H=1.1)
    q.update(over)
    return base_scene(**q)


def gauss_renders(p: dict) -> dict[str, dict]:
    """Flat mirror, bare bump and cloaked bump versions of one scene (Fig. 4 a, b, c)."""
    return {
        "mirror": dict(p, mirror=FLAT, cloak=0),
        "bare": dict(p, mirror=GAUSS, cloak=0),
        "cloak": dict(p, mirror=GAUSS, cloak=1),
    }


def config_small(precision: int = FP64) -> dict:
    """64 x 64, 1 sample per pixel (pixel centres), RK4 h = Lambda/200."""
    return base_scene(width=64, height=64, spp=1, seed=1, precision=precision)


def config_main(precision: int = FP32) -> dict:
    """512 x 512, 4 samples per pixel (2 x 2 stratified, seed 2), RK4 h = Lambda/200."""
    return base_scene(width=512, height=512, spp=4, seed=2, precision=precision)


def config_hd(extent: float = 8.0, A: float = 0.04, tex_size: int = 2048, precision: int = FP32) -> dict:
    """1920 x 1080, 16 samples per pixel, Dormand-Prince RK45, value-noise background."""
    rtol = 1e-5 if precision == FP32 else 1e-7
    return base_scene(width=1920, height=1080, spp=16, seed=3, E=extent, A=A, integrator=DP45,
                      rtol=rtol, atol=rtol, background=TEXTURE, tex_size=tex_size,
                      precision=precision)


def batch_scenes(count: int = 64, seed: int = 4, precision: int = FP32) -> list[dict]:
    """Scenes of uneven size and parameters drawn from the seed: side in
    {128, 256, 512, 1024}, spp in {1, 4, 16}, A ~ U[0.01, 0.04] Lambda,
    Lambda ~ U[0.5, 2], elevation ~ U[10, 60] deg, azimuth ~ U[0, 90] deg,
    E = 8 Lambda, H = 2 Lambda."""
    rng = np.random.default_rng([seed, 0xBA7C])
    out = []
    for i in range(count):
        side = int(rng.choice([128, 256, 512, 1024]))
        spp = int(rng.choice([1, 4, 16]))
        lam = float(rng.uniform(0.5, 2.0))
        A = float(rng.uniform(0.01, 0.04))
        p = base_scene(width=side, height=side, spp=spp, seed=seed * 1000 + i, scene_id=i,
                       elev_deg=float(rng.uniform(10.0, 60.0)), azim_deg=float(rng.uniform(0.0, 90.0)),
                       A=A, precision=precision)
        out.append(scale_scene(p, lam))
    return out


def serving_requests(count: int, seed: int = 5, rate: float = 200.0, max_side: int = 2048,
                     min_side: int = 256, max_spp: int = 64, precision: int = FP32) -> list[tuple[float, dict]]:
    """Poisson arrivals (mean `rate` per second) of render requests with side
    log-uniform in [min_side, max_side], spp log-uniform in [1, max_spp]
    (rounded), scene parameters as for the batched scenes.  Returns
    (arrival time in seconds, scene) pairs."""
    rng = np.random.default_rng([seed, 0x5E7E])
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        side = int(round(math.exp(rng.uniform(math.log(min_side), math.log(max_side)))))
        spp = max(1, int(round(math.exp(rng.uniform(0.0, math.log(max_spp))))))
        lam = float(rng.uniform(0.5, 2.0))
        p = base_scene(width=side, height=side, spp=spp, seed=seed * 100000 + i, scene_id=i,
                       elev_deg=float(rng.uniform(10.0, 60.0)), azim_deg=float(rng.uniform(0.0, 90.0)),
                       A=float(rng.uniform(0.01, 0.04)), precision=precision)
        out.append((t, scale_scene(p, lam)))
    return out


def pixel_subset(height: int, width: int, count: int, seed: int) -> np.ndarray:
    """Seeded random subset of flat pixel indices (sorted, without repeats)."""
    rng = np.random.default_rng([seed, 0x5A3B])
    n = height * width
    if count >= n:
        return np.arange(n, dtype=np.int64)
    return np.sort(rng.choice(n, size=count, replace=False)).astype(np.int64)
