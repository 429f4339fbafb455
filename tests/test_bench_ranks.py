"""The multi-process path of bench.py on CPU (gloo, two ranks).

Every rank renders the whole workload (independent replicas, no collective on
the data path), so the only cross-rank logic is the timing: the slowest rank's
time and the job's total ray count give the whole-job throughput, and rank 0
alone prints the line.  The reference arm under torchrun runs on rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = 100.0 + 37.5 * rank          # this rank's timed total in ms
        slowest = bench.max_over_ranks(dist, mine, "cpu")
        ms, value = bench.whole_job(1_000_000, world, slowest, 4)
        q.put((rank, slowest, ms, value))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, ms, value in out:
        assert slowest == 137.5              # rank 1's time, seen by both ranks
        assert ms == pytest.approx(137.5 / 4)
        # two replicas of 1e6 rays per step in the slowest rank's step time
        assert value == pytest.approx(2 * 1_000_000 / (137.5 / 4 * 1e-3) / 1e6)


def test_whole_job_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.whole_job(3_151_872, 1, 212.36, 10)
    assert ms == pytest.approx(21.236)
    assert value == pytest.approx(3_151_872 / 0.021236 / 1e6)


def test_reference_arm_torchrun_two_ranks():
    """Under torchrun with two ranks the reference arm prints one line, from rank 0."""
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--ref-pixels", "2"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["n_gpus"] == 2
    assert line["value"] > 0 and line["unit"] == "Mrays/s"
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
