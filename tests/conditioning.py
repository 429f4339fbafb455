"""Conditioning of single rays under the FP64 oracle (helpers, no tests).

FP32 carries about 1e-7 relative rounding into every quantity of a ray once
the ray reaches the scene.  How far a ray's exit moves when its direction is
turned by a small angle where it reaches the scene tells which rays FP32
arithmetic can resolve at all: the parity bars of the FP32 path are stated
over all rays and, separately, over the rays that the oracle itself finds
well conditioned."""
import numpy as np


def scene_entry(p, org, d):
    """Parameter t at which the camera ray org + t d first reaches the scene:
    the cloak box (slab test) or the band y <= A of the grating, whichever
    comes first; None if it reaches neither."""
    ts = []
    if d[1] < 0.0:
        ts.append((max(p["A"], 1e-6 * p["Lambda"]) - org[1]) / d[1])
    if p["cloak"]:
        lo = np.array([-p["E"] / 2, -p["A"], -p["E"] / 2])
        hi = np.array([p["E"] / 2, p["H"] - p["A"], p["E"] / 2])
        with np.errstate(divide="ignore", invalid="ignore"):
            t1, t2 = (lo - org) / d, (hi - org) / d
        tn, tf = np.minimum(t1, t2).max(), np.maximum(t1, t2).min()
        if tn <= tf and tn > 0:
            ts.append(tn)
    ts = [t for t in ts if t > 0]
    return min(ts) if ts else None


def turned_exits(orc, sc, p, i, j, s, angle, ref=None):
    """Largest change of exit direction (rad) and position over four turns of
    the camera ray of sample s of pixel (i, j) by `angle` rad (two
    perpendicular axes, both signs) where it reaches the scene; infinite when
    a turn changes the path (bounce count or status).  (0, 0) for rays that
    never reach the scene.  `ref`: the unturned record, if already traced."""
    org, d = orc.camera_dir(sc, i, j, s)
    t = scene_entry(p, org, d)
    if t is None:
        return 0.0, 0.0
    start = org + 0.999999 * t * d
    if ref is None:
        ref, _ = orc.trace_from(sc, start, d)
    a = np.cross(d, [0.0, 1.0, 0.0])
    a /= np.linalg.norm(a)
    b = np.cross(d, a)
    dd = dp = 0.0
    for e in (a, b, -a, -b):
        d2 = d + angle * e
        d2 /= np.linalg.norm(d2)
        r, _ = orc.trace_from(sc, start, d2)
        if r["bounces"] != ref["bounces"] or r["status"] != ref["status"]:
            return np.inf, np.inf
        dd = max(dd, float(np.linalg.norm(np.asarray(r["dir"]) - np.asarray(ref["dir"]))))
        dp = max(dp, float(np.abs(np.asarray(r["pos"]) - np.asarray(ref["pos"])).max()))
    return dd, dp
