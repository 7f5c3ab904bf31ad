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


# ----------------------------------------- block filter shared out by blocks
def _exact_filter_pieces(lat, U, Up, kappa, colour_mask):
    """Oracle-backed compute and decision steps of the partitioned filter: the
    exact block log-ratio of every block is computed on its own (dense LU of
    its Dirichlet operator), so a rank's values do not depend on which other
    blocks it holds."""
    import numpy as np
    from oracle import accept, dirac

    pos_of = lat.dd_pos[[lat.block_sites_of(b)[0] for b in range(lat.nblocks)]] // lat.block_sites

    def compute_range(pos0, npos):
        out = np.zeros(lat.nblocks)
        for b in range(lat.nblocks):
            if pos0 <= pos_of[b] < pos0 + npos:
                out[b] = 2.0 * (dirac.logabsdet(dirac.dense_dirichlet_block(Up, lat, kappa, b))
                                - dirac.logabsdet(dirac.dense_dirichlet_block(U, lat, kappa, b)))
        return out

    def decide(ln_b):
        acc, _ = accept.block_accept(ln_b, 7, 3, colour_mask, lat.block_colour)
        return acc, accept.restore_rejected_blocks(Up, U, lat, acc)

    return compute_range, decide


def _filter_inputs():
    """A proposal that changes every active link by a large random rotation
    (some blocks of each colour are then rejected)."""
    from oracle import geometry
    from paper_1112_1243_gb300 import synthetic
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.4, 5)
    R = synthetic.random_gauge(dims, 1.0, 22)
    Up = U.copy()
    Up[lat.active] = R[lat.active] @ U[lat.active]
    return lat, U, Up


def _filter_worker(rank, world, port, out):
    import numpy as np
    from paper_1112_1243_gb300 import partition
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lat, U, Up = _filter_inputs()
        res = {}
        for cm in (1, 2, 3):
            compute_range, decide = _exact_filter_pieces(lat, U, Up, 0.12, cm)

            def reduce_sum(v):
                t = torch.from_numpy(np.ascontiguousarray(v))
                dist.all_reduce(t, op=dist.ReduceOp.SUM)
                return t.numpy()

            ln_b, (acc, Unew) = partition.filter_partition_step(rank, world, lat.nblocks, cm, compute_range,
                                                                 reduce_sum, decide)
            res[cm] = (ln_b.tobytes(), acc.tobytes(), Unew.tobytes())
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_block_ranges_cover_the_selected_colours():
    from paper_1112_1243_gb300 import partition
    for nb in (2, 16, 512):
        for cm in (1, 2, 3):
            for world in (1, 2, 3, 8):
                r = partition.block_ranges(nb, cm, world)
                assert len(r) == world
                first = nb // 2 if cm == 2 else 0
                count = nb if cm == 3 else nb // 2
                pos = first
                for p0, n in r:
                    assert p0 == pos and n >= 0
                    pos += n
                assert pos == first + count
                assert max(n for _, n in r) - min(n for _, n in r) <= 1


def test_two_gloo_ranks_partitioned_filter_equals_single_rank():
    """Both ranks of a partitioned (exact) block filter end with the
    single-rank log-ratios, decisions and restored field, bit for bit."""
    import numpy as np
    from paper_1112_1243_gb300 import partition
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_filter_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    lat, U, Up = _filter_inputs()
    for cm in (1, 2, 3):
        compute_range, decide = _exact_filter_pieces(lat, U, Up, 0.12, cm)
        ln_b, (acc, Unew) = partition.filter_partition_step(0, 1, lat.nblocks, cm, compute_range, lambda v: v, decide)
        assert np.any(ln_b != 0) and not np.all(acc)
        for r in range(world):
            assert res[r][cm] == (ln_b.tobytes(), acc.tobytes(), Unew.tobytes()), (r, cm)
