"""Oracle pins for 3-D rays in the cloak and total reflection at its side
faces (Sec. 3: the index of the grating cloak, Eq. 1, depends on x and y
only; at a face of the finite cloak the tangential momentum is kept, and a
ray whose tangential momentum exceeds the index of the air outside is
reflected)."""
import numpy as np
import pytest

from paper_1012_5107_gb300 import inputs


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle as o
    o.build()
    return o


@pytest.fixture(scope="module")
def scene(orc):
    p = inputs.three_renders(inputs.config_main(precision=inputs.FP64))["cloak"]
    return orc.Scene(p), p


@pytest.mark.parametrize("method", [0, 1])
def test_3d_ray_moves_like_its_planar_part(orc, scene, method):
    """The index does not depend on z, so a 3-D ray's (x, y, p_x, p_y) evolve
    exactly as those of the same ray with p_z = 0, while z advances by p_z per
    unit of the ray parameter and p_z stays constant.  A force or an index
    that wrongly took z or p_z into account fails this."""
    sc, p = scene
    h = p["h"]
    rng = np.random.default_rng(4)
    for _ in range(8):
        x, y = rng.uniform(-0.5, 0.5), rng.uniform(0.06, 0.8)
        n = orc.index(sc, x, y)[2]
        ang = rng.uniform(0.0, 2.0 * np.pi)
        pz = rng.uniform(0.2, 0.6) * n
        pxy = np.sqrt(n * n - pz * pz)
        s3 = np.array([x, y, 0.25, pxy * np.cos(ang), pxy * np.sin(ang), pz])
        s2 = s3.copy()
        s2[5] = 0.0
        a3 = orc.integrate_fixed(sc, s3, h, 40, method=method)
        a2 = orc.integrate_fixed(sc, s2, h, 40, method=method)
        assert np.array_equal(a3[:, [0, 1, 3, 4]], a2[:, [0, 1, 3, 4]])
        tau = h * np.arange(1, 41)
        assert np.allclose(a3[:, 2], 0.25 + pz * tau, rtol=0.0, atol=1e-13)
        assert np.all(a3[:, 5] == pz)
        assert np.all(a2[:, 2] == 0.25)


@pytest.mark.parametrize("axis", [0, 2])
def test_total_reflection_at_a_side_face(orc, scene, axis):
    """A ray just inside the +x (or +z) face of the box, where the index is
    about 1.28, with a tangential momentum of 1.1 (more than the index 1 of the
    air): it meets the face, keeps its position there, and leaves it with the
    normal momentum component reversed and the two tangential ones unchanged,
    then goes on inside the box."""
    sc, p = scene
    E2 = p["E"] / 2.0
    x0, y0 = 4.0 - 1e-3 if axis == 0 else 0.0, 0.06       # x = 4 Lambda: a crest of the grating
    n = orc.index(sc, x0, y0)[2]
    assert 1.2 < n < 1.35
    pt = 1.1                                                # |p_t| > 1: no refraction into air
    pn = np.sqrt(n * n - pt * pt)
    X = np.array([x0, y0, 0.0])
    mom = np.array([pn, 0.0, pt]) if axis == 0 else np.array([pt, 0.0, pn])
    if axis == 2:
        X[2] = E2 - 1e-3
    rec, traj = orc.trace_from(sc, X, mom, medium=1, traj_cap=400)
    # the event: two consecutive records at the same point, the second one reflected
    idx = [q for q in range(1, len(traj)) if np.array_equal(traj[q, :3], traj[q - 1, :3])]
    assert idx, "no reflection recorded"
    q = idx[0]
    before, after = traj[q - 1], traj[q]
    assert abs(before[axis] - E2) < 1e-9                    # on the face
    assert after[3 + axis] == pytest.approx(-before[3 + axis], rel=0, abs=1e-15)
    for a in range(3):
        if a != axis:
            assert after[3 + a] == before[3 + a]
    assert before[3 + axis] > 0.0
    # it goes on inside the box after the reflection
    assert traj[q + 1, axis] < E2
