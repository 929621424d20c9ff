"""bench.py's multi-rank path on the CPU: two gloo ranks (replicas of the
scan, no collective on the data path) agree on the slowest rank's time, and
the whole-job rate counts every rank's SNPs."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank 1 is the slow replica; only rank 0 ran the end-to-end leg
        t_local = [2.0, 3.5][rank]
        e2e_local = [4.0, None][rank]
        t, e2e = bench.max_over_ranks(t_local, e2e_local, dist, torch, "cpu")
        out.put((rank, t, e2e))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert got == [(0, 3.5, 4.0), (1, 3.5, 4.0)]
    # 2 replicas x 10^6 SNPs x 3 steps in 3.5 s
    assert bench.whole_job_rate(2, 1_000_000, 3, 3.5) == pytest.approx(2e6 * 3 / 3.5)


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(1.5, None, None, torch, "cpu") == (1.5, None)
