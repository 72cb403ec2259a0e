"""The benchmark harness's multi-rank logic on CPU (two gloo ranks): each rank solves its own replica,
the step time is the slowest rank's, the value counts every rank's DOF; the reference arm runs on
rank 0 only."""

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
torch = pytest.importorskip("torch")

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, ms: list, out) -> None:
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    got = bench.max_over_ranks(ms[rank], dist, "cpu")
    out.put((rank, got, bench.whole_job_value(1000, world, got)))
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ms = [10.0, 12.5]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [12.5, 12.5]
    assert all(abs(r[2] - 2 * 1000 / 0.0125) < 1e-6 for r in res)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_value(4096 * 16384, 1, 41.0) == pytest.approx(4096 * 16384 / 0.041)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
