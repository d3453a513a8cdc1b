"""The benchmark's N>1 path on the CPU: one replica per rank (the method has no exchange step on one
instance), ranks joined over gloo on 127.0.0.1.  Every rank gets the slowest rank's time, the
whole-job value counts the points of all ranks within that time, and the reference arm runs on
rank 0 only: the other ranks exit 0 without work or output.  The batched workload's independent
instances are shared out over the ranks: every instance on exactly one rank, loads balanced to
within the largest instance, one rank keeping the original order."""
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


def _rank(rank, world, port, local_ms, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(local_ms[rank], world, "cpu")
        value = bench.job_throughput(world, 1 << 20, ms, 10)
        out.put((rank, ms, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    local_ms = [31.5, 27.25]  # rank 1 is faster; both report rank 0's time
    procs = [ctx.Process(target=_rank, args=(r, 2, port, local_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for _, ms, value in got:
        assert ms == 31.5
        # 2 replicas x 2^20 points per step, 10 steps in 31.5 ms
        assert value == pytest.approx(2 * (1 << 20) / (3.15e-3), rel=1e-15)


def test_one_rank_is_its_own_max():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(1, 1000, 20.0, 4) == pytest.approx(1000 / 5e-3, rel=1e-15)


@pytest.mark.parametrize("rank", [1, 3])
def test_reference_arm_on_other_ranks_exits_without_work(rank):
    env = dict(os.environ, WORLD_SIZE="4", RANK=str(rank), LOCAL_RANK=str(rank),
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "4",
                        "--steps", "2", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_returns_nothing_off_rank_0():
    import argparse
    import bench
    assert bench.run_reference(argparse.Namespace(steps=1, warmup=3), 1) is None


def _sizes(k=512, seed=3):
    import numpy as np
    return [int(v) for v in np.exp(np.random.default_rng(seed).uniform(np.log(1e3), np.log(2e5), k))]


def test_one_rank_keeps_every_instance_in_order():
    import bench
    sizes = _sizes()
    assert bench.shard_instances(sizes, 1, 0) == list(range(len(sizes)))


@pytest.mark.parametrize("world", [2, 3, 4, 8])
def test_shards_partition_and_balance(world):
    import bench
    sizes = _sizes()
    shards = [bench.shard_instances(sizes, world, r) for r in range(world)]
    flat = sorted(i for sh in shards for i in sh)
    assert flat == list(range(len(sizes)))              # every instance exactly once
    assert all(sh == sorted(sh) for sh in shards)      # ascending on each rank
    loads = [sum(sizes[i] for i in sh) for sh in shards]
    assert max(loads) - min(loads) <= max(sizes)       # largest-first greedy bound
    assert shards == [bench.shard_instances(sizes, world, r) for r in range(world)]  # deterministic


def _shard_rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = _sizes(64, 4)
        mine = bench.shard_instances(sizes, world, rank)
        pts = sum(sizes[i] for i in mine)
        ms = bench.max_over_ranks(pts * 1e-4, world, "cpu")  # time grows with the rank's points
        out.put((rank, mine, pts, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_sharded_batch_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = _sizes(64, 4)
    assert sorted(got[0][1] + got[1][1]) == list(range(64))
    assert got[0][2] + got[1][2] == sum(sizes)
    slowest = max(got[0][2], got[1][2]) * 1e-4
    assert got[0][3] == pytest.approx(slowest, rel=1e-12) and got[1][3] == pytest.approx(slowest, rel=1e-12)
