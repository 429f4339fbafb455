"""The render server: continuous batching under a ray-state budget, with
the requests in a device-resident ring that a running launch takes work
from.  Every result equals a render of the same scene alone (the scenes are
mixed into shared launches and overlap on the device)."""
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


def requests(count, seed):
    out = []
    for t, p in inputs.serving_requests(count, seed=seed, max_side=64, min_side=16, max_spp=16):
        out.append((t, p))
    return out


def wait_all(server, tickets, limit_s=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets) and time.time() - t0 < limit_s:
        for t in tickets:
            if t not in res:
                r = server.poll(t, timeout_us=2000)
                if r is not None:
                    res[t] = r
    return res


def test_results_equal_alone(rt):
    import torch
    reqs = requests(12, seed=5)
    alone = []
    for _, p in reqs:
        sc = rt.Scene(p)
        img = torch.zeros(sc.shape, dtype=torch.float32, device="cuda")
        sc.render(img)
        alone.append(img)
    torch.cuda.synchronize()
    server = rt.Server(budget_bytes=1 << 30, max_inflight=3)
    outs, tickets = [], []
    t_start = time.time()
    for (t_arr, p) in reqs:
        while time.time() - t_start < t_arr:        # the seeded Poisson arrivals
            time.sleep(0.0005)
        out = torch.full(rt.Scene(p).shape, -1.0, dtype=torch.float32, device="cuda")
        outs.append(out)
        tickets.append(server.submit(p, out))
    res = wait_all(server, tickets)
    assert len(res) == len(tickets)
    for t in tickets:
        assert res[t]["status"] == 0 and res[t]["latency_ms"] >= res[t]["queue_ms"] >= 0
    torch.cuda.synchronize()
    for a, b in zip(alone, outs):
        assert torch.equal(a, b)
    st = server.stats()
    assert st["completed"] == len(reqs) and st["bytes_in_use"] == 0 and st["queued"] == 0
    server.close()


def test_budget_admission_and_busy(rt):
    import torch
    reqs = requests(6, seed=7)
    server = rt.Server(budget_bytes=1, max_inflight=2)
    out = torch.zeros((64, 64, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(rt.RtError) as e:
        server.submit(reqs[0][1], out)
    assert e.value.code == rt.RT_EBUSY
    server.close()
    # a budget that holds one request at a time still serves every request
    biggest = max(rt.request_bytes(p) for _, p in reqs)
    assert biggest == max(p["width"] * p["height"] * (p["spp"] * 76 + 16) for _, p in reqs)
    server = rt.Server(budget_bytes=biggest, max_inflight=2)
    outs = [torch.zeros(rt.Scene(p).shape, dtype=torch.float32, device="cuda") for _, p in reqs]
    tickets = [server.submit(p, o) for (_, p), o in zip(reqs, outs)]
    assert server.stats()["bytes_in_use"] <= biggest
    res = wait_all(server, tickets)
    assert all(r["status"] == 0 for r in res.values()) and len(res) == len(reqs)
    server.close()


def test_poll_semantics(rt):
    import torch
    server = rt.Server(budget_bytes=1 << 28, max_inflight=1)
    with pytest.raises(rt.RtError):
        server.poll(12345)
    p = inputs.base_scene(width=32, height=32, spp=4, precision=0)
    out = torch.zeros((32, 32, 3), dtype=torch.float32, device="cuda")
    t = server.submit(p, out)
    r = None
    for _ in range(20000):
        r = server.poll(t, timeout_us=1000)
        if r is not None:
            break
    assert r is not None and r["rays"] == 32 * 32 * 4
    with pytest.raises(rt.RtError):            # a finished ticket is reported once
        server.poll(t)
    with pytest.raises(rt.RtError) as e:       # invalid descriptors are refused at submission
        server.submit(dict(p, Lambda=-1.0), out)
    assert e.value.code == rt.RT_EINVAL
    server.close()


def test_close_with_work_pending(rt):
    import torch
    server = rt.Server(budget_bytes=1 << 28, max_inflight=1)
    outs = []
    for _, p in requests(8, seed=11):
        o = torch.zeros(rt.Scene(p).shape, dtype=torch.float32, device="cuda")
        outs.append(o)
        server.submit(p, o)
    server.close()                               # waits for flights, fails the rest
    torch.cuda.synchronize()


def test_running_launch_takes_new_requests(rt):
    """A small request submitted while a large one is on the GPU finishes
    first: the running launch takes its samples as lanes free up, instead of
    the request waiting for the large one to end."""
    import torch
    big = inputs.base_scene(width=1024, height=1024, spp=16, seed=21, scene_id=1, precision=0)
    small = inputs.base_scene(width=48, height=40, spp=4, seed=22, scene_id=2, precision=0)
    ref = torch.zeros((40, 48, 3), dtype=torch.float32, device="cuda")
    sc = rt.Scene(small)
    sc.render(ref)
    torch.cuda.synchronize()
    server = rt.Server(budget_bytes=4 << 30, max_inflight=2)
    out_big = torch.zeros((1024, 1024, 3), dtype=torch.float32, device="cuda")
    out_small = torch.full((40, 48, 3), -1.0, dtype=torch.float32, device="cuda")
    tb = server.submit(big, out_big)
    time.sleep(0.01)                                    # the large request is running
    ts = server.submit(small, out_small)
    rs = None
    for _ in range(20000):
        rs = server.poll(ts, timeout_us=1000)
        if rs is not None:
            break
    assert rs is not None and rs["status"] == 0
    assert server.poll(tb) is None                      # the large one is still running
    rb = wait_all(server, [tb])[tb]
    assert rb["status"] == 0 and rb["latency_ms"] > rs["latency_ms"] + 10.0
    torch.cuda.synchronize()
    assert torch.equal(out_small, ref)
    server.close()


def test_ring_wraps_around(rt):
    """More requests than the ring has slots (1024), each equal to its render alone."""
    import torch
    n = 1100
    ps = [inputs.base_scene(width=8, height=6, spp=1 + (q % 3), seed=100 + q, scene_id=q, precision=0)
          for q in range(n)]
    server = rt.Server(budget_bytes=1 << 28, max_inflight=2)
    outs = [torch.zeros((6, 8, 3), dtype=torch.float32, device="cuda") for _ in ps]
    tickets = [server.submit(p, o) for p, o in zip(ps, outs)]
    res = wait_all(server, tickets, limit_s=300.0)
    assert len(res) == n and all(r["status"] == 0 for r in res.values())
    torch.cuda.synchronize()
    for q in (0, 1, 513, 1023, 1024, 1025, n - 1):
        sc = rt.Scene(ps[q])
        ref = torch.zeros((6, 8, 3), dtype=torch.float32, device="cuda")
        sc.render(ref)
        torch.cuda.synchronize()
        assert torch.equal(outs[q], ref), q
    st = server.stats()
    assert st["completed"] == n and st["in_flight"] == 0 and st["bytes_in_use"] == 0
    server.close()


def test_small_request_passes_one_waiting_for_budget(rt):
    """Admission under a budget that holds one large request and one small
    one: a second large request must wait for the first, but a small request
    submitted after it is admitted at once (it passes the waiting one) and
    finishes before it; every result equals the render alone."""
    import torch
    big1 = inputs.base_scene(width=1024, height=1024, spp=16, seed=31, scene_id=1, precision=0)
    big2 = inputs.base_scene(width=1024, height=1024, spp=16, seed=32, scene_id=2, precision=0)
    small = inputs.base_scene(width=48, height=40, spp=4, seed=33, scene_id=3, precision=0)
    budget = rt.request_bytes(big1) + rt.request_bytes(small)
    assert rt.request_bytes(big1) + rt.request_bytes(big2) > budget
    ref = torch.zeros((40, 48, 3), dtype=torch.float32, device="cuda")
    sc = rt.Scene(small)
    sc.render(ref)
    torch.cuda.synchronize()
    server = rt.Server(budget_bytes=budget, max_inflight=2)
    outs = [torch.zeros((1024, 1024, 3), dtype=torch.float32, device="cuda") for _ in range(2)]
    out_small = torch.full((40, 48, 3), -1.0, dtype=torch.float32, device="cuda")
    t1 = server.submit(big1, outs[0])
    t2 = server.submit(big2, outs[1])
    ts = server.submit(small, out_small)
    res = wait_all(server, [t1, t2, ts])
    assert len(res) == 3 and all(r["status"] == 0 for r in res.values())
    r1, r2, rs = res[t1], res[t2], res[ts]
    # the second large request waited for the first one's budget; the small
    # one did not wait for either
    assert r2["queue_ms"] > 0.5 * r1["latency_ms"]
    assert rs["queue_ms"] < 0.25 * r1["latency_ms"]
    assert rs["latency_ms"] < r1["latency_ms"] < r2["latency_ms"]
    torch.cuda.synchronize()
    assert torch.equal(out_small, ref)
    server.close()
