"""Failure detection without a GPU fault: the wavefront loop's bounded waits.

Every wait of a block on its work queues gives up after a bounded number of
attempts, counts the timeout and lets the launch end; rt_scene_stats then
reports RT_ETIMEDOUT.  Here a scene starts every block with its queue lock
held (rt_scene_set_wait_limit), so that every wait runs out: the launch must
end by itself within a short time, report the timeouts, and leave the context
usable, so that the next normal render of the same scene gives the same image
as before."""
import time

import numpy as np
import pytest

from paper_1012_5107_gb300 import inputs

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


@pytest.mark.parametrize("precision", [0, 1])
def test_bounded_wait_runs_out_and_context_survives(rt, precision):
    import torch
    p = inputs.base_scene(width=40, height=24, spp=4, seed=3, precision=precision)
    sc = rt.Scene(p)
    sc.set_launch(3, 0)                           # the wavefront loop
    ref = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
    sc.render(ref)
    torch.cuda.synchronize()
    st = sc.stats()
    assert st["sched_timeouts"] == 0 and st["rays"] == 40 * 24 * 4

    sc.set_wait_limit(64, hold_lock=True)
    rgb = torch.full(sc.shape, -1.0, dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    sc.render(rgb)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 10.0
    with pytest.raises(rt.RtError) as e:
        sc.stats()
    assert e.value.code == rt.RT_ETIMEDOUT
    st = sc.stats(check=False)
    assert st["rc"] == rt.RT_ETIMEDOUT
    # every warp of every block gave up its first wait: no sample was started
    assert st["sched_timeouts"] == sc.get_launch()["grid"] * 8
    assert st["rays"] == 0
    assert (rgb.cpu().numpy() == -1.0).all()

    sc.set_wait_limit(0, hold_lock=False)         # back to the default bound
    out = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
    sc.render(out)
    torch.cuda.synchronize()
    st = sc.stats()
    assert st["sched_timeouts"] == 0 and st["rays"] == 40 * 24 * 4
    assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())
    sc.close()


def test_wait_limit_is_validated(rt):
    sc = rt.Scene(inputs.base_scene(width=8, height=8, spp=1, precision=0))
    for bad in (-1, (1 << 24) + 1):
        with pytest.raises(rt.RtError) as e:
            sc.set_wait_limit(bad)
        assert e.value.code == rt.RT_EINVAL
    sc.set_wait_limit(1 << 24)
    sc.close()
