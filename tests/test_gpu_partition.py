"""The block filter shared out by block ranges (paper_1112_1243_gb300.partition):
the ranges of two ranks, computed one after the other on one GPU (nothing
waits on anything), summed and decided, reproduce dd_block_filter's
log-ratios, decisions and restored field bit for bit (its persistent
per-block form, the same per-block solves)."""
import numpy as np
import pytest

from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,block,cm,n", [((8, 8, 8, 8), (4, 4, 4, 4), 3, 2), ((8, 8, 8, 8), (4, 4, 4, 4), 2, 1),
                                            ((16, 16, 16, 16), (8, 8, 8, 8), 3, 2)])
def test_two_ranges_equal_the_whole_filter(dims, block, cm, n):
    api = lib_api()
    from paper_1112_1243_gb300 import partition
    h = api.dd_init(dims, block, 0.13, max_rhs=n)
    api.dd_set_tuning(h, filter_masked=0)
    U = dev(synthetic.random_gauge(dims, 0.3, 2))
    Up = U.clone()
    api.dd_gauge_update(h, Up, 3, 5.3, 1, 0, 11, 3)
    ref_U = Up.clone()
    ln_ref, acc_ref = api.dd_block_filter(h, U, ref_U, cm, api.DD_FILTER_STOCHASTIC, n, 99, 5)
    world = 2
    ranks = []
    for rank in range(world):
        def compute_range(pos0, npos):
            return api.dd_block_ratios_range(h, U, Up, pos0, npos, n, 99, 5)
        ranks.append((rank, compute_range))
    parts = [cr(*partition.block_ranges(h.nfine, cm, world)[r]).clone() for r, cr in ranks]
    total = parts[0] + parts[1]
    for p in parts:
        assert np.count_nonzero(host(p)) > 0            # both ranks hold blocks
    Unew = Up.clone()
    acc = api.dd_block_accept(h, U, Unew, cm, total, 99, 5)
    assert host(total).tobytes() == host(ln_ref).tobytes()
    assert np.array_equal(host(acc), host(acc_ref))
    assert host(Unew).tobytes() == host(ref_U).tobytes()
    assert api.dd_status(h)[0] == 0
    # a single rank through the product wrapper (no process group)
    Un2 = Up.clone()
    ln1, acc1 = partition.partitioned_block_filter(h, U, Un2, cm, n, 99, 5)
    assert host(ln1).tobytes() == host(ln_ref).tobytes()
    assert host(Un2).tobytes() == host(ref_U).tobytes()
