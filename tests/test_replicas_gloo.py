"""The bench's multi-GPU path is replicas only (the subcycle runs whole on
each GPU; no data-path collective): two gloo ranks on the CPU check the
host logic it uses -- the barrier, the max over ranks of the timed region,
the whole-job value -- and that only rank 0 runs the reference arm."""
import json
import os
import subprocess
import sys

import pytest

import bench

torch = pytest.importorskip("torch")


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms = 10.0 + 5.0 * rank          # rank 1 is the slower one
    worst = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    v = bench.replica_value(world, 205379, 200, 10, worst)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, worst, v))


def test_two_gloo_ranks_take_the_slowest_time():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    # two replicas of 205379 cells x 200 subcycles x 10 steps in 15 ms
    assert out[0][2] == pytest.approx(2 * 205379 * 200 * 10 / 15e-3)
    assert out[0][2] == out[1][2]


def test_single_process_needs_no_collective():
    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert bench.replica_value(1, 100, 200, 10, 1000.0) == pytest.approx(100 * 200 * 10)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=bench.ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""
