"""The multi-GPU path of bench.py is replicas only: each rank runs the whole
workload and the only exchange is the max over ranks of the step time.  Two
gloo ranks on the CPU check that reduction, the whole-job rate and that only
rank 0 of the reference arm does work."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    ms = bench.ranks_max(100.0 + 50.0 * rank, world, "cpu")
    q.put((rank, ms, bench.job_rate(1e9, ms, world)))
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks_and_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in out:
        assert ms == 150.0                       # the slower rank's time on every rank
        assert rate == pytest.approx(2 * 1e9 / 0.150)


def test_world_one_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.ranks_max(7.5, 1, "cpu") == 7.5
    assert bench.job_rate(10.0, 1000.0, 1) == pytest.approx(10.0)


def test_reference_arm_on_a_nonzero_rank_does_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
