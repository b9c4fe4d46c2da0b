"""Host logic of bench.py's multi-rank run, on CPU with gloo (world size 2).

Each rank solves its own replica of the cube (no exchange between cubes), so
the whole-job rate is the units of all ranks over the slowest rank's time.
The reference arm runs on rank 0 only; other ranks exit 0 without work.
"""

import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        own = [0.25, 0.40][rank]
        slowest = bench.max_over_ranks(own, dist, "cpu")
        rate = bench.whole_job_rate(1000, slowest, world)
        out.put((rank, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_whole_job_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(out.get() for _ in range(world))
    for rank, slowest, rate in res:
        assert slowest == 0.40, rank
        assert rate == pytest.approx(2 * 1000 / 0.40)


def test_single_process_keeps_its_own_time():
    assert bench.max_over_ranks(0.5) == 0.5
    assert bench.whole_job_rate(10, 2.0, 1) == 5.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
