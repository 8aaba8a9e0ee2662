"""The multi-process side of bench.py on CPU (gloo, world size 2): ranks
run independent replicas with disjoint Philox keys, the job is timed by the
slowest rank (max over ranks), the value aggregates every rank's units, and
under torchrun only rank 0 runs the reference arm."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    seeds = bench.rank_seeds(rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds.tolist())
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, dist, "cpu")
    value = bench.aggregate(world, 8_192_000 * 4, ms_max * 1e-3)
    dist.barrier()
    out.put((rank, gathered, ms_max, value))
    dist.destroy_process_group()


def test_two_ranks_disjoint_seeds_and_max_time():
    world, port = 2, 29517
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, ms_max, value in res:
        a, b = set(gathered[0]), set(gathered[1])
        assert len(a) == len(b) == 8 and not (a & b)
        assert ms_max == 15.0
        assert value == pytest.approx(2 * 8_192_000 * 4 / 0.015)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert np.array_equal(bench.rank_seeds(0), np.arange(8, dtype=np.uint64) + 2001)
    assert bench.aggregate(1, 100.0, 2.0) == 50.0


def test_reference_arm_runs_on_rank_zero_only():
    """Launched as rank 1 of 2, the reference arm exits 0 at once and prints
    nothing (rank 0 alone times the oracle and prints the line)."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
