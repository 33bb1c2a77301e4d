"""Multi-rank host logic of bench.py, on CPU over gloo with world size 2.

On the GPU each rank runs an independent replica of the decomposition (the
path has no data exchange); the ranks meet only to take the slowest rank's
time, and the whole-job rate counts every rank's work over that time.  The
uneven batch instead shards by matrix, every rank computing the same
assignment.  The reference arm runs on rank 0 alone.
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


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    local_ms = [10.0, 25.0][rank]
    mx = bench.max_over_ranks(local_ms, world)
    rate = bench.whole_job_rate(world, 4, 3e9, mx)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mx, rate))


def test_slowest_rank_time_and_whole_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, mx, rate in res:
        assert mx == 25.0                                     # the slower rank's time
        assert rate == pytest.approx(2 * 4 * 3e9 / 0.025 / 1e9)   # both ranks' work


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(1, 10, 4.58e10, 59.1) == pytest.approx(10 * 4.58e10 / 0.0591 / 1e9)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""


def _batch_works():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1301_4438_gb300 import workloads as W
    bt = W.batch_2000()
    return bench, [bench.fops(m, n, r) for m, n, r in zip(bt.ms, bt.ns, bt.rs)]


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_batch_shards_cover_the_batch_once_and_balance(world):
    """Over several GPUs the uneven batch shards by matrix (no data exchange):
    the shards partition the 2000 matrices, and the longest-first assignment
    keeps every rank's work within one matrix of the mean."""
    bench, works = _batch_works()
    shards = [bench.batch_shard(works, r, world) for r in range(world)]
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(len(works)))
    loads = [sum(works[i] for i in s) for s in shards]
    assert max(loads) - min(loads) <= max(works)
    assert max(loads) <= sum(works) / world + max(works)
    for s in shards:   # each shard is handed out largest first
        assert [works[i] for i in s] == sorted((works[i] for i in s), reverse=True)


def _shard_rank_main(rank, world, port, q):
    import torch.distributed as dist
    bench, works = _batch_works()
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    mine = bench.batch_shard(works, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    slowest = bench.max_over_ranks(sum(works[i] for i in mine), world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, gathered, slowest))


def test_batch_shards_agree_across_gloo_ranks():
    """Each rank computes its own shard; gathered over two gloo ranks, the
    shards partition the batch and the slowest rank carries the larger load."""
    bench, works = _batch_works()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, g0, s0), (_, g1, s1) = res
    assert g0 == g1
    assert sorted(g0[0] + g0[1]) == list(range(len(works)))
    assert s0 == s1 == max(sum(works[i] for i in g0[0]), sum(works[i] for i in g0[1]))
