"""bench.py's multi-rank bookkeeping (replicas, one per GPU): the job's time is
the slowest rank's and its rate counts every rank's units.  Two gloo ranks on
the CPU; the reference arm prints from rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # rank 1 is slower
    slow = bench.slowest_rank_ms(ms, world)
    out.put((rank, slow, bench.whole_job_rate(1e9, world, slow)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, slow, rate in res:
        assert slow == 15.0
        assert rate == pytest.approx(2 * 1e9 / 0.015)


def test_single_rank_needs_no_process_group():
    assert bench.slowest_rank_ms(7.5, 1) == 7.5
    assert bench.whole_job_rate(3e9, 1, 1000.0) == pytest.approx(3e9)


def test_reference_arm_prints_from_rank_zero_only(tmp_path):
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
