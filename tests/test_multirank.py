"""The multi-GPU path of the benchmark is replicas (one independent chain per
rank, no data-path collective): the host logic is covered here with two
gloo ranks on the CPU: every rank gets the slowest rank's time, the job
rate counts the units of all ranks, and the ranks' chains use distinct
seeds."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = 100.0 + 50.0 * rank          # rank 1 is the slowest
        t_max = bench.max_over_ranks(t_local, world)
        rate = bench.job_rate(12, world, t_max)
        seeds = bench.replica_seeds(bench.CONFIGS["c5"], rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        out[rank] = (t_max, rate, tuple(gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        t_max, rate, seeds = res[r]
        assert t_max == 150.0
        assert abs(rate - 12 * 2 / 0.15) < 1e-9
        assert len(set(seeds)) == world           # distinct (field, chain) seeds per rank
        assert len({s[0] for s in seeds}) == world and len({s[1] for s in seeds}) == world


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(123.0, 1) == 123.0
    assert bench.job_rate(12, 1, 2000.0) == 6.0
