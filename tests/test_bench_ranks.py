"""The benchmark's N > 1 path on the CPU: two `gloo` ranks in separate processes.

Every rank runs an independent replica of the factor-and-solve step (there is no exchange in the
path), so the job's time is the slowest rank's and its work is the sum over ranks.  These tests
drive the benchmark's own cross-rank helpers through a real world-size-2 process group, and check
that the reference arm does its CPU work on rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, ms_by_rank, units_by_rank):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        env = bench._rank_env()
        bench._barrier()
        ms, units = bench._job_time(ms_by_rank[rank], units_by_rank[rank], "cpu")
        bench._barrier()
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"env": env, "ms": ms, "units": units}, f)


def _spawn(tmp_path, ms_by_rank, units_by_rank):
    world = len(ms_by_rank)
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), ms_by_rank, units_by_rank),
                       nprocs=world, join=True, start_method="spawn")
    return [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]


def test_job_time_is_max_time_and_summed_units(tmp_path):
    res = _spawn(tmp_path, [812.5, 967.25], [48, 48])
    for r, x in enumerate(res):
        assert x["env"] == [2, r, r]
        # every rank sees the same whole-job figures: the slower rank's time, both ranks' RHS
        assert x["ms"] == 967.25
        assert x["units"] == 96


def test_job_time_uneven_units(tmp_path):
    # the batched workload can give the ranks different totals; the sum is exact
    res = _spawn(tmp_path, [3.0, 1.5], [1024, 7])
    assert all(x["ms"] == 3.0 and x["units"] == 1031 for x in res)


def test_job_time_without_process_group_passes_through():
    sys.path.insert(0, ROOT)
    import bench

    assert not dist.is_initialized()
    assert bench._job_time(12.5, 16, "cpu") == (12.5, 16)
    bench._barrier()  # no process group: a no-op


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def _shard_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        allp = W.config(3)
        mine = bench._shard(allp, world, rank)
        shares = [None] * world
        dist.all_gather_object(shares, [(p.problem, p.n) for p in mine])
        # the job's work is every rank's right-hand sides: the whole batch's
        _, units = bench._job_time(1.0, sum(p.nrhs for p in mine), "cpu")
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, f"shard{rank}.json"), "w") as f:
        json.dump({"mine": [(p.problem, p.n) for p in mine], "shares": shares, "units": units,
                   "all": [(p.problem, p.n) for p in allp]}, f)


@pytest.mark.parametrize("world", [2, 3])
def test_batched_problems_are_sharded_across_ranks(tmp_path, world):
    mp.start_processes(_shard_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"shard{r}.json")) for r in range(world)]
    allp = [tuple(x) for x in res[0]["all"]]
    assert len(allp) == 64
    seen = []
    for r, x in enumerate(res):
        mine = [tuple(v) for v in x["mine"]]
        assert mine == allp[r::world]  # problem i on rank i mod world
        assert [[tuple(v) for v in sh] for sh in x["shares"]] == [allp[q::world] for q in range(world)]
        seen += mine
        assert x["units"] == sum(1 for _ in allp)  # one RHS per problem, summed over the ranks
    assert sorted(seen) == sorted(allp) and len(set(seen)) == len(allp)  # disjoint, and the union is the batch
