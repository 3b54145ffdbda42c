"""Host logic of the multi-GPU path, on CPU with the gloo backend.

Every problem is independent, so N GPUs run N replicas of the workload with
no collective on the data path; the benchmark only takes the slowest rank's
time and reports the whole job's rate.  These tests run that logic with two
gloo ranks, and check that under torchrun only rank 0 of the reference arm
prints.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank measured a different time; everyone must see the slowest
    t = bench.max_over_ranks(1.0 + rank, world)
    rate = bench.job_rate(2.0e9, t, world)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, rate))


def test_two_gloo_ranks_agree_on_slowest_time_and_job_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]
    # 2 GFLOP per rank on 2 ranks over the slowest 2 s: 2 GFLOP/s for the job
    assert all(abs(r[2] - 2.0) < 1e-12 for r in res)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_rate(1e9, 0.5, 1) == 2.0


@pytest.mark.parametrize("rank", [1])
def test_reference_arm_other_ranks_exit_quietly(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
