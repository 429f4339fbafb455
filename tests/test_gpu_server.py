"""The render server: continuous batching under a ray-state budget.  Every
result equals a render of the same scene alone (the scenes are mixed into
shared batch launches and overlap on the device)."""
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
