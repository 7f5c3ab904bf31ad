"""The allocation-free entry point dd_block_ratios_noalloc, for callers that
cannot allocate device memory (graph capture in global mode, host
applications that own all device memory, loops that cannot afford the
synchronisation of cudaMalloc), must give the block log-ratios that the
workspace-based dd_block_filter gives for one factor.

Collected last (file name), so that a run stopping at the first failure has
run every other test first.  Works alone in a fresh process and after the
other tests: the scratch array is set up on the first call and reused.
Tolerance: 1e-8 absolute, the block log-ratio tolerance of the other tests
(both paths run the same arithmetic; the results are in fact expected to be
identical).
"""
import numpy as np
import pytest

from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api

pytestmark = pytest.mark.gpu


def test_noalloc_block_ratios_match_block_filter():
    api = lib_api()
    import torch
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.13
    h = api.dd_init(dims, block, kappa, max_rhs=1, tol_block=1e-12)
    U = dev(synthetic.random_gauge(dims, 0.3, 2))
    Up = U.clone()
    api.dd_gauge_update(h, Up, 3, 5.3, 1, 0, 11, 3)
    nblocks = h.nblocks
    for cm in (3, 2, 1):
        Up_filter = Up.clone()  # dd_block_filter restores rejected blocks in place
        ln_ref, _ = api.dd_block_filter(h, U, Up_filter, cm, api.DD_FILTER_STOCHASTIC, 1, 99, 5)
        ref = host(ln_ref)
        assert np.any(ref != 0)
        for call in range(2):
            ln = torch.full((nblocks,), float("nan"), dtype=torch.float64, device="cuda")
            api.dd_block_ratios_noalloc(dims, block, kappa, -1, cm, U, Up, 99, 5, 1e-12, ln)
            got = host(ln)
            assert np.all(np.isfinite(got)), (cm, call)
            assert np.max(np.abs(got - ref)) < 1e-8, (cm, call, np.max(np.abs(got - ref)))


def test_noalloc_reports_unconverged_blocks_as_nan():
    """A block whose FP64 refinement cannot reach tol_block within the fixed
    12 cycles gets ln_b = NaN (the entry point has no status word); blocks of
    the unselected colour keep 0.  Bounded: 12 cycles of at most 2000 FP32
    iterations per block."""
    api = lib_api()
    import torch
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.13
    h = api.dd_init(dims, block, kappa, max_rhs=1)
    U = dev(synthetic.random_gauge(dims, 0.3, 2))
    Up = U.clone()
    api.dd_gauge_update(h, Up, 3, 5.3, 1, 0, 11, 3)
    colour = np.array([sum(((b // (2 ** 0)) % 2, (b // 2) % 2, (b // 4) % 2, (b // 8) % 2)) % 2
                       for b in range(h.nblocks)])
    ln = torch.zeros((h.nblocks,), dtype=torch.float64, device="cuda")
    api.dd_block_ratios_noalloc(dims, block, kappa, -1, 2, U, Up, 99, 5, 1e-30, ln)
    got = host(ln)
    assert np.all(np.isnan(got[colour == 1])), got
    assert np.all(got[colour == 0] == 0.0), got
    # the next call with a reachable tolerance is unaffected
    ln2 = torch.full((h.nblocks,), float("nan"), dtype=torch.float64, device="cuda")
    api.dd_block_ratios_noalloc(dims, block, kappa, -1, 2, U, Up, 99, 5, 1e-12, ln2)
    assert np.all(np.isfinite(host(ln2)))
