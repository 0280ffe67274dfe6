"""The multi-GPU path is replicas only (the sweep does not shard): these CPU
tests run its host logic as two gloo ranks, and check that the reference arm
does its work on rank 0 alone."""

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    from paper_2108_07549_gb300 import replicas

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = 1.5 + rank  # rank 1 is the slowest
        s = replicas.slowest(mine, world, device="cpu")
        out[rank] = (s, replicas.job_throughput(1e9, s, world))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_job_throughput_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    with ctx.Manager() as manager:
        out = manager.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1] == (2.5, 2 * 1e9 / 2.5)


def test_single_rank_needs_no_process_group():
    from paper_2108_07549_gb300 import replicas

    assert replicas.slowest(3.0, 1) == 3.0
    assert replicas.job_throughput(10.0, 2.0, 1) == 5.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--workload", "knn2500_k500"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
