"""Multi-process host logic of bench.py on CPU (gloo, world size 2).

With N GPUs the bench runs one replica of the workload per rank (the
near-field pass of one box has no exchange step here); only the timing is
reduced across ranks.  The batched configuration instead shards its 64
independent boxes over the ranks, which exchange only their pair totals and
times.  These tests cover those reductions, the box assignment, the
whole-job rate and the reference arm's rank rule without a GPU.
"""
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


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(times[rank])
    dist.barrier()
    out[rank] = t
    dist.destroy_process_group()


def test_timing_is_the_max_over_ranks():
    world, port = 2, _free_port()
    times = [1234.5, 987.25]
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, times, out), nprocs=world, join=True)
    assert out[0] == out[1] == max(times)


def test_whole_job_rate_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(10 ** 12, 1, 1000.0) == pytest.approx(1000.0)
    assert bench.whole_job_rate(10 ** 12, 4, 1000.0) == pytest.approx(4000.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def _batched_worker(rank, world, port, pairs, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.shard_boxes(64, rank, world)
    out[rank] = (mine, bench.batched_job(pairs[rank], times[rank], world))
    dist.barrier()
    dist.destroy_process_group()


def test_batched_boxes_shard_over_ranks_with_only_totals_exchanged():
    world, port = 2, _free_port()
    pairs, times = [3 * 10 ** 11, 10 ** 11], [210.0, 95.5]
    out = mp.Manager().dict()
    mp.spawn(_batched_worker, args=(world, port, pairs, times, out), nprocs=world, join=True)
    (b0, j0), (b1, j1) = out[0], out[1]
    assert sorted(b0 + b1) == list(range(64)) and not set(b0) & set(b1)     # a partition of the boxes
    assert b0 == list(range(0, 64, 2)) and b1 == list(range(1, 64, 2))
    assert j0 == j1
    total, ms, rate = j0
    assert total == sum(pairs) and ms == max(times)
    assert rate == pytest.approx(sum(pairs) / (max(times) * 1e-3) / 1e9)


def test_shard_boxes_covers_every_box_for_any_world():
    sys.path.insert(0, ROOT)
    import bench
    for world in (1, 3, 8, 64, 100):
        got = sorted(i for r in range(world) for i in bench.shard_boxes(64, r, world))
        assert got == list(range(64))

