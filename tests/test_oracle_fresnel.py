"""Pins for the oracle's Fresnel weights, referenced cloak and dielectric plate
(Sec. 3: Snell and Fresnel at the cloak interface, rays Fresnel-reflected
more than once neglected; Sec. 4 and Figs. 5-7: the index profile divided by
n_min, and a homogeneous plate of index 1/n_min on the flat mirror as the
ideal reference)."""
import math

import numpy as np
import pytest

from paper_1012_5107_gb300 import inputs


# ---------------------------------------------------------------------------
# Fresnel reflectance (unpolarised)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n1,n2", [(1.0, 1.5), (1.0, 1.37), (1.6, 1.0), (1.0, 2.2)])
def test_fresnel_normal_incidence(orc, n1, n2):
    assert abs(orc.fresnel(n1, n2, 1.0) - ((n1 - n2) / (n1 + n2)) ** 2) < 1e-15


@pytest.mark.parametrize("n1,n2", [(1.0, 1.5), (1.37, 1.0), (1.0, 2.2)])
def test_fresnel_brewster_angle(orc, n1, n2):
    """At Brewster's angle (tan = n2/n1) the p wave is not reflected and the s
    reflection amplitude is (n1^2 - n2^2)/(n1^2 + n2^2)."""
    thb = math.atan2(n2, n1)
    rs = (n1 * n1 - n2 * n2) / (n1 * n1 + n2 * n2)
    assert abs(orc.fresnel(n1, n2, math.cos(thb)) - 0.5 * rs * rs) < 1e-14


@pytest.mark.parametrize("n1,n2", [(1.0, 1.5), (1.0, 1.25)])
def test_fresnel_reciprocity_and_limits(orc, n1, n2):
    for th1 in np.linspace(0.0, 1.5, 13):
        th2 = math.asin(n1 * math.sin(th1) / n2)
        a, b = orc.fresnel(n1, n2, math.cos(th1)), orc.fresnel(n2, n1, math.cos(th2))
        assert abs(a - b) < 1e-13 and 0.0 <= a <= 1.0
    assert orc.fresnel(n1, n2, 1e-9) > 0.999999                   # grazing incidence
    thc = math.asin(n1 / n2)                                       # beyond the critical angle
    assert orc.fresnel(n2, n1, math.cos(thc + 0.01)) == 1.0


# ---------------------------------------------------------------------------
# The dielectric plate on the flat mirror (Figs. 5-7 (a))
# ---------------------------------------------------------------------------
def _plate_scene(orc, fresnel):
    p = inputs.base_scene(mirror=0, cloak=0, flags=orc.FLAG_PLATE | (orc.FLAG_FRESNEL if fresnel else 0),
                          E=40.0, precision=1)
    return orc.Scene(p), p


@pytest.mark.parametrize("fresnel", [False, True])
def test_plate_parallel_displacement(orc, fresnel):
    """A ray through the plate leaves parallel to its mirror image, displaced
    along the plate by 2 t tan(theta_t), t = plate thickness; with Fresnel
    weights the path keeps T_in T_out = T^2 (reciprocity)."""
    sc, p = _plate_scene(orc, fresnel)
    kA = 2 * math.pi * p["A"] / p["Lambda"]
    npl = 1.0 + kA
    top = -p["A"] + p["H"]
    d = np.array([0.3, -0.8, 0.2]); d /= np.linalg.norm(d)
    X0 = np.array([-1.0, top + 3.0, 0.5])
    rec, w = orc.trace_paths(sc, X0, d)
    r0 = rec[0]
    assert r0["status"] == 0 and r0["bounces"] == 1
    dexp = d * np.array([1, -1, 1])
    assert np.abs(r0["dir"] - dexp).max() < 1e-14
    t_in = (X0[1] - top) / -d[1]
    Xe = X0 + t_in * d                                         # entry point on the top face
    pt = np.array([d[0], 0.0, d[2]])
    shift = 2 * top * pt / math.sqrt(npl ** 2 - pt @ pt)
    assert np.abs(r0["pos"] - (Xe + shift)).max() < 1e-12
    R = orc.fresnel(1.0, npl, -d[1])
    if not fresnel:
        assert len(w) == 1 and w[0] == 1.0
        return
    # first path T^2; entry reflection R (leaves from the entry point along the
    # mirrored direction); internal reflection at the exit T R, which leaves
    # after a second trip with T R T
    assert len(w) == 3
    assert abs(w[0] - (1 - R) ** 2) < 1e-14
    assert abs(w[1] - R) < 1e-14 and np.abs(rec[1]["pos"] - Xe).max() < 1e-12
    assert np.abs(rec[1]["dir"] - dexp).max() < 1e-14
    assert abs(w[2] - (1 - R) * R * (1 - R)) < 1e-14
    assert np.abs(rec[2]["pos"] - (Xe + 2 * shift)).max() < 1e-12
    assert rec[2]["bounces"] == 2


def test_plate_scene_needs_the_flat_mirror(orc):
    p = inputs.base_scene(mirror=1, cloak=0, flags=orc.FLAG_PLATE, precision=1)
    with pytest.raises(ValueError):
        orc.render_pixels(orc.Scene(p), [0])


# ---------------------------------------------------------------------------
# The referenced cloak: n / n_min (Sec. 4, Figs. 5-7)
# ---------------------------------------------------------------------------
def test_referenced_index_profile(orc):
    p = inputs.base_scene(A=3.0 / (16.0 * math.pi), precision=1)
    kA = 2 * math.pi * p["A"] / p["Lambda"]
    ref = orc.Scene(dict(p, flags=orc.FLAG_REFERENCED))
    unref = orc.Scene(p)
    xs = np.linspace(-0.5, 0.5, 41)
    ys = 0.2 + 0.5 * np.abs(xs)
    a, b = orc.index(ref, xs, ys), orc.index(unref, xs, ys)
    assert np.allclose(a[:, 2], (1 + kA) * b[:, 2], rtol=1e-14)
    assert np.allclose(a[:, 3:5], (1 + kA) * b[:, 3:5], rtol=1e-14, atol=1e-14)
    # on the grating at a trough (x = Lambda/2) the referenced index is exactly 1 (Fig. 1 (a))
    xi = 0.5 * p["Lambda"]
    ys_ = orc.trochoid(unref, [xi])[0, 1]
    assert abs(orc.index(ref, xi, ys_)[2] - 1.0) < 1e-12
    assert abs((1 + kA) - 1.375) < 1e-12                   # n = 1/n_min = 1.375 for A = 3/(16 pi)


def test_referenced_cloak_traces_the_same_curves(orc):
    """Dividing every index inside the cloak by n_min leaves its rays' curves
    unchanged (Sec. 4): a ray started inside with the same direction exits at
    the same point in the same direction."""
    base = inputs.base_scene(integrator=1, rtol=1e-11, atol=1e-11, precision=1)
    kA = 2 * math.pi * base["A"] / base["Lambda"]
    unref = orc.Scene(base)
    ref = orc.Scene(dict(base, flags=orc.FLAG_REFERENCED))
    X = np.array([0.3, 1.2, -0.4])
    d = np.array([0.25, -0.9, 0.1]); d /= np.linalg.norm(d)
    n0 = orc.index(unref, X[0], X[1])[2]
    ra, _ = orc.trace_from(unref, X, n0 * d, medium=1)
    rb, _ = orc.trace_from(ref, X, (1 + kA) * n0 * d, medium=1)
    # the first exit from the box is the same point; the refraction into air
    # then differs because the air keeps n = 1
    _, traj_a = orc.trace_from(unref, X, n0 * d, medium=1, traj_cap=100000)
    _, traj_b = orc.trace_from(ref, X, (1 + kA) * n0 * d, medium=1, traj_cap=100000)
    ea, eb = traj_a[-1], traj_b[-1]
    assert np.abs(ea[:3] - eb[:3]).max() < 1e-8
    da = ea[3:] / np.linalg.norm(ea[3:])
    db = eb[3:] / np.linalg.norm(eb[3:])
    assert np.abs(da - db).max() < 1e-8
    assert ra["bounces"] == rb["bounces"]


# ---------------------------------------------------------------------------
# Fresnel weights in a cloak render
# ---------------------------------------------------------------------------
def test_fresnel_weights_in_the_cloak(orc):
    """Weights of a sample's paths: the first path loses a Fresnel reflection
    at each crossing, each branch carries one; what is lost is only the
    twice-reflected light, of order R^2."""
    p = inputs.base_scene(flags=orc.FLAG_FRESNEL | orc.FLAG_REFERENCED, precision=1)
    sc = orc.Scene(p)
    o, d = orc.camera_dir(sc, 20, 32, 0)
    rec, w = orc.trace_paths(sc, o, d)
    assert len(w) >= 2 and w[0] < 1.0
    assert 1.0 - 0.02 < w.sum() <= 1.0 + 1e-12
    # the first branch is the reflection at the entry through the top face:
    # weight R(1 -> n(entry), cos = -d_y), leaving along the mirrored direction
    top = -p["A"] + p["H"]
    Xe = o + (top - o[1]) / d[1] * d
    assert abs(Xe[0]) < p["E"] / 2 and abs(Xe[2]) < p["E"] / 2
    n_e = orc.index(sc, Xe[0], Xe[1])[2]
    assert abs(w[1] - orc.fresnel(1.0, n_e, -d[1])) < 1e-12
    assert np.abs(rec[1]["pos"] - Xe).max() < 1e-9
