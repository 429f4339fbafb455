"""Pins for the oracle's ray dynamics (Sec. 3, Eqs. 9-11) and integrators."""
import math

import numpy as np
import pytest

from paper_1012_5107_gb300 import inputs


def _sc(orc, **kw):
    return orc.Scene(inputs.base_scene(**kw))


def _start(orc, sc, x, y, ang_deg, pz=0.0):
    n = orc.index(sc, x, y)[2]
    d = np.array([math.cos(math.radians(ang_deg)), math.sin(math.radians(ang_deg)), 0.0])
    d[:2] *= math.sqrt(max(1.0 - pz * pz, 0.0))
    d[2] = pz
    return np.array([x, y, 0.0]), n * d


def test_straight_rays_without_grating(orc):
    """A = 0 makes n = 1 everywhere: the acceleration vanishes (Sec. 3)."""
    sc = _sc(orc, A=0.0, E=100.0, H=4.0)
    X, p = _start(orc, sc, 0.3, 3.0, -35.0, pz=0.2)
    rec, traj = orc.trace_from(sc, X, p, medium=1, traj_cap=5000)
    pre = traj[: np.argmin(traj[:, 1]) + 1]
    d = p / np.linalg.norm(p)
    rel = pre[:, :3] - X
    perp = rel - np.outer(rel @ d, d)
    assert np.abs(perp).max() < 1e-12
    assert np.abs(pre[:, 3:] - p).max() == 0.0


def test_hamiltonian_and_pz_invariants(orc):
    sc = _sc(orc, A=0.05)
    X, p = _start(orc, sc, 0.1, 0.4, -5.0, pz=0.4)
    s0 = np.concatenate([X, p])
    tr = orc.integrate_fixed(sc, s0, 0.005, 300, method=0)
    n = orc.index(sc, tr[:, 0], tr[:, 1])[:, 2]
    ham = (tr[:, 3:] ** 2).sum(1) - n ** 2
    assert np.abs(ham).max() < 1e-10
    assert (tr[:, 5] == p[2]).all()           # p_z is conserved exactly (Sec. 3: grad n has no z part)
    assert np.allclose(tr[:, 2], X[2] + p[2] * 0.005 * np.arange(1, 301), atol=1e-13)


@pytest.mark.parametrize("method,order", [(0, 4), (1, 5), (2, 4)])
def test_integrator_order(orc, method, order):
    """Fixed-step error shrinks as h^order (pins the RK4 and Dormand-Prince tableaus)."""
    sc = _sc(orc, A=0.06)
    X, p = _start(orc, sc, 0.2, 0.35, -10.0, pz=0.3)
    s0 = np.concatenate([X, p])
    T = 0.4
    ref = orc.integrate_fixed(sc, s0, T / 800, 800, method=1)[-1]
    errs = []
    for m in (10, 20, 40):
        errs.append(np.abs(orc.integrate_fixed(sc, s0, T / m, m, method=method)[-1] - ref).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    expect = 2.0 ** order
    assert 0.6 * expect < r1 < 1.6 * expect, errs
    assert 0.6 * expect < r2 < 1.6 * expect, errs


def test_time_form_eq11_traces_the_same_curve(orc):
    """Integrate Eq. 11 literally in physical time (c0 = 1, |v| = c0/n) with
    scipy and compare the curve with the oracle's tau-parametrised one."""
    solve_ivp = pytest.importorskip("scipy.integrate").solve_ivp
    sc = _sc(orc, A=0.06)
    X, p = _start(orc, sc, -0.3, 0.45, -12.0, pz=0.0)
    s0 = np.concatenate([X, p])
    tr = orc.integrate_fixed(sc, s0, 0.002, 250, method=1)

    def rhs(t, u):
        r, v = u[:3], u[3:]
        g = orc.index(sc, r[0], r[1])
        n, gn = g[2], g[3:6]
        a = ((v @ v) * gn - 2 * (gn @ v) * v) / n
        return np.concatenate([v, a])

    n0 = orc.index(sc, X[0], X[1])[2]
    v0 = p / np.linalg.norm(p) / n0
    sol = solve_ivp(rhs, (0, 1.2), np.concatenate([X, v0]), method="DOP853", rtol=1e-12, atol=1e-13,
                    dense_output=True)
    tt = np.linspace(0, sol.t[-1], 40001)
    xs, ys = sol.sol(tt)[0], sol.sol(tt)[1]
    assert np.all(np.diff(xs) > 0)
    inside = tr[:, 0] < xs[-1]
    y_interp = np.interp(tr[inside, 0], xs, ys)
    assert np.abs(y_interp - tr[inside, 1]).max() < 2e-8
    # speed stays c0/n along the Eq. 11 solution
    vv = sol.sol(tt[::1000])[3:]
    nn = orc.index(sc, sol.sol(tt[::1000])[0], sol.sol(tt[::1000])[1])[:, 2]
    assert np.abs(np.linalg.norm(vv, axis=0) * nn - 1).max() < 1e-9


def test_2d_cloak_is_a_flat_mirror_in_virtual_space(orc):
    """For p_z = 0 the conformal map w = z + i W0/k turns the cloak's curved rays
    into straight lines reflected at v = 0 (Sec. 2; exactness in 2D, Sec. 5)."""
    A = 0.06
    k = 2 * math.pi
    # tight adaptive steps: the pin is on the physics, not on RK4's h = Lambda/200 error
    sc = _sc(orc, A=A, H=6.0, E=1000.0, integrator=1, rtol=1e-12, atol=1e-12)
    for ang in (-30.0, -55.0, -80.0):
        X, p = _start(orc, sc, 0.17, 5.5, ang)
        rec, traj = orc.trace_from(sc, X, p, medium=1, traj_cap=20000)
        assert rec["bounces"] == 1 and rec["status"] == 0
        W = orc.index(sc, traj[:, 0], traj[:, 1])
        w = traj[:, 0] + 1j * traj[:, 1] + 1j * (W[:, 0] + 1j * W[:, 1]) / k
        ih = int(np.argmin(np.abs(w.imag)))
        assert abs(w[ih].imag) < 1e-12
        d_in = p[0] + 1j * p[1]
        d_in /= abs(d_in)
        d_out = d_in.conjugate()
        pre, post = w[: ih + 1], w[ih:]
        dist_pre = np.abs(((pre - w[0]) * d_in.conjugate()).imag)
        dist_post = np.abs(((post - w[ih]) * d_out.conjugate()).imag)
        assert dist_pre.max() < 1e-9 and dist_post.max() < 1e-9, (dist_pre.max(), dist_post.max())
        dout = np.asarray(rec["dir"])
        assert abs(dout[0] - d_out.real) < 1e-9 and abs(dout[1] - d_out.imag) < 1e-9


def test_rk4_converges_and_agrees_with_dp45(orc):
    base = inputs.base_scene(width=16, height=16, spp=1)
    pix = np.arange(16 * 16)
    dirs = {}
    for name, over in [("h1", dict(h=0.01)), ("h2", dict(h=0.005)), ("h4", dict(h=0.0025)),
                       ("dp", dict(integrator=1, rtol=1e-10, atol=1e-10))]:
        sc = orc.Scene(dict(base, **over))
        _, rec = orc.render_pixels(sc, pix, records=True)
        dirs[name] = rec
    ok = (dirs["h4"]["bounces"] == dirs["dp"]["bounces"]) & (dirs["h1"]["bounces"] == dirs["h4"]["bounces"])
    assert ok.mean() > 0.95
    e1 = np.abs(dirs["h1"]["dir"] - dirs["h4"]["dir"])[ok].max()
    e2 = np.abs(dirs["h2"]["dir"] - dirs["h4"]["dir"])[ok].max()
    assert e1 / max(e2, 1e-300) > 8.0          # ~ (2^4 - 1)/(1 - 2^-4) * ... for fourth order
    assert np.abs(dirs["h4"]["dir"] - dirs["dp"]["dir"])[ok].max() < 1e-7
    assert np.abs(dirs["h4"]["pos"] - dirs["dp"]["pos"])[ok].max() < 1e-6


# ---------------------------------------------------------------------------
# The tracer's time form of Eq. 11 (integrator 2: RK4 in t, state (r, v))
# ---------------------------------------------------------------------------
def test_time_form_tracer_matches_tau_form(orc):
    """A ray started inside the cloak leaves at the same point in the same
    direction whether the tracer integrates Eq. 11 in t or the Hamiltonian
    form in tau (the same curves, Sec. 3); the step sizes differ, so they
    agree to the integration error."""
    from paper_1012_5107_gb300 import inputs
    base = inputs.base_scene(A=0.05, h=1.0 / 800, precision=1)
    tau = orc.Scene(base)
    tform = orc.Scene(dict(base, integrator=2))
    X = np.array([0.21, 0.9, -0.3])
    d = np.array([0.3, -0.85, 0.12]); d /= np.linalg.norm(d)
    n0 = orc.index(tau, X[0], X[1])[2]
    ra, _ = orc.trace_from(tau, X, n0 * d, medium=1)
    rb, _ = orc.trace_from(tform, X, n0 * d, medium=1)
    assert ra["bounces"] == rb["bounces"] >= 1 and ra["status"] == rb["status"]
    assert np.abs(ra["pos"] - rb["pos"]).max() < 1e-9
    assert np.abs(ra["dir"] - rb["dir"]).max() < 1e-9


def test_time_form_invariants(orc):
    """Along the time-form solution the speed stays c0/n and n^2 v_z (the
    conserved momentum p_z of the z-translation invariance) stays fixed."""
    from paper_1012_5107_gb300 import inputs
    sc = orc.Scene(inputs.base_scene(A=0.05, h=1.0 / 400, integrator=2, precision=1))
    X = np.array([-0.37, 1.1, 0.2])
    d = np.array([0.2, -0.9, 0.35]); d /= np.linalg.norm(d)
    n0 = orc.index(sc, X[0], X[1])[2]
    _, traj = orc.trace_from(sc, X, n0 * d, medium=1, traj_cap=20000)
    assert len(traj) > 100
    seg = traj[: np.argmax(np.abs(np.diff(traj[:, 4])) > 0.05)]     # up to the first reflection
    n = orc.index(sc, seg[:, 0], seg[:, 1])[:, 2]
    speed = np.linalg.norm(seg[:, 3:], axis=1)
    assert np.abs(speed * n - 1.0).max() < 1e-10
    pz = n * n * seg[:, 5]
    assert np.abs(pz - pz[0]).max() < 1e-10
