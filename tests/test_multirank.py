"""The replicas path of the bench on CPU ranks (gloo, world size 2): every
rank reports the slowest rank's time, the job's throughput counts the units of
all ranks, the replicas draw different problems, and under two ranks the
reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    value, t = bench.job_throughput(0.5 + rank, 1000.0, world)
    seed = bench.replica_seed(2, rank)
    phantom_sum = float(workloads.phantom_2d(32, seed, 5).sum())
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, value, t, seed, phantom_sum))


def test_two_replicas_report_the_slowest_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, value, t, seed, _ in out:
        assert t == 1.5                          # max over ranks of 0.5 and 1.5
        assert value == pytest.approx(2 * 1000.0 / 1.5)
    assert out[0][3] != out[1][3] and out[0][4] != out[1][4]   # different problems


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.job_throughput(2.0, 10.0, 1) == (5.0, 2.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                        "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
