"""The benchmark's multi-rank logic (replicas, one process per GPU) on CPU: two gloo ranks
on 127.0.0.1 check the slowest-rank time reduction and the whole-job rate, and that the
reference arm does its work on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env()[:2] == (rank, world)
        dist.barrier()
        t = bench.max_over_ranks(times[rank], world)
        rate = bench.whole_job_rate(1000, world, 10, t)
        out.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    times = [0.25, 0.75]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == 0.75                       # every rank sees the slowest rank's time
        assert rate == pytest.approx(1000 * 2 * 10 / 0.75)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(0.5, 1) == 0.5
    assert bench.whole_job_rate(4096, 1, 100, 2.0) == 4096 * 100 / 2.0


def test_reference_arm_skips_non_zero_ranks(capsys):
    class Args:
        workload, cpu_seconds, steps, warmup = "film_small", 1.0, 1, 1
    assert bench.run_reference(Args(), rank=1, world=2) is None
    assert capsys.readouterr().out == ""
