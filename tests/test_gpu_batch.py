"""The block filters of three lattices with different block shapes (4^4, 6^4,
8^4) in one persistent launch (dd_block_filter_batch) give exactly what the
per-lattice dd_block_filter gives (same streams, same per-item arithmetic,
deterministic reductions), and the 6^4 blocks agree with the oracle.
"""
import numpy as np
import pytest

from oracle import accept, estimator, geometry, heatbath
from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api

pytestmark = pytest.mark.gpu

LATTICES = [((8, 8, 8, 8), (4, 4, 4, 4), 1),      # DD_ACTIVE_PAPER
            ((12, 12, 12, 12), (6, 6, 6, 6), 1),
            ((16, 16, 16, 16), (8, 8, 8, 8), 2)]  # DD_ACTIVE_INNER6


def _setup(api, n):
    hs, Us, Ups = [], [], []
    for k, (dims, block, mode) in enumerate(LATTICES):
        h = api.dd_init(dims, block, 0.13, active_mode=mode, max_rhs=n)
        U = dev(synthetic.random_gauge(dims, 0.3, 20 + k))
        Up = U.clone()
        api.dd_gauge_update(h, Up, 3, 5.3, 1, 0, 31, 7)
        hs.append(h)
        Us.append(U)
        Ups.append(Up)
    return hs, Us, Ups


def test_batch_equals_per_lattice_filters():
    api = lib_api()
    n = 4
    hs, Us, Ups = _setup(api, n)
    Ups_batch = [u.clone() for u in Ups]
    ln_bs, accs = api.dd_block_filter_batch(hs, Us, Ups_batch, 3, n, 99, 5)
    for k, h in enumerate(hs):
        Up_single = Ups[k].clone()
        ln_ref, acc_ref = api.dd_block_filter(h, Us[k], Up_single, 3, api.DD_FILTER_STOCHASTIC, n, 99, 5)
        assert np.array_equal(host(ln_bs[k]), host(ln_ref)), k
        assert np.array_equal(host(accs[k]), host(acc_ref)), k
        assert np.array_equal(host(Ups_batch[k]), host(Up_single)), k
        assert np.all(host(ln_bs[k]) != 0)
        assert api.dd_status(h)[0] == 0


def test_batch_6x4_blocks_against_oracle():
    """One factor on the 12^4 lattice with 6^4 blocks, compared with the oracle."""
    api = lib_api()
    dims, block = (12, 12, 12, 12), (6, 6, 6, 6)
    lat = geometry.Lattice(dims, block, active_mode="paper")
    U = synthetic.random_gauge(dims, 0.3, 21)
    Up, _ = heatbath.gauge_update(U, lat, 5.3, 1, 0, 31, 7)
    h8 = api.dd_init((8, 8, 8, 8), (4, 4, 4, 4), 0.13, max_rhs=1)
    h12 = api.dd_init(dims, block, 0.13, active_mode=1, max_rhs=1)
    U8 = dev(synthetic.random_gauge((8, 8, 8, 8), 0.3, 20))
    U8p = U8.clone()
    api.dd_gauge_update(h8, U8p, 3, 5.3, 1, 0, 31, 7)
    Upd = dev(Up)
    ln_bs, accs = api.dd_block_filter_batch([h12, h8], [dev(U), U8], [Upd, U8p], 3, 1, 99, 5)
    ref = estimator.block_ln_ratios(U, Up, lat, 0.13, 1, 99, 5, colour_mask=3, tol=1e-13)
    got = host(ln_bs[0])
    assert np.max(np.abs(got - ref)) < 1e-8, np.max(np.abs(got - ref))
    racc, lu = accept.block_accept(ref, 99, 5, 3, lat.block_colour)
    clear = np.abs(lu - ref) > 1e-8
    assert np.array_equal(host(accs[0]).astype(bool)[clear], racc[clear])


def test_batch_filter_graph_replay_matches_eager():
    """The uneven-block batch recorded once as a CUDA graph on the first
    handle and replayed: the same log-ratios, decisions and restored fields
    as the eager call, bit for bit."""
    api = lib_api()
    import torch
    cases = [((8, 8, 8, 8), (4, 4, 4, 4)), ((8, 8, 8, 8), (2, 2, 2, 2)), ((12, 12, 12, 12), (6, 6, 6, 6))]
    n = 2
    hs, Us, Ups = [], [], []
    for k, (dims, block) in enumerate(cases):
        h = api.dd_init(dims, block, 0.13, max_rhs=n)
        U = dev(synthetic.random_gauge(dims, 0.3, 40 + k))
        Up = U.clone()
        api.dd_gauge_update(h, Up, 3, 5.3, 1, 0, 7, 2)
        hs.append(h)
        Us.append(U)
        Ups.append(Up)
    work = [u.clone() for u in Ups]
    ln = [torch.zeros(h.nblocks, dtype=torch.float64, device="cuda") for h in hs]
    acc = [torch.zeros(h.nblocks, dtype=torch.uint8, device="cuda") for h in hs]
    api.dd_block_filter_batch(hs, Us, work, 3, n, 11, 5, ln, acc)
    eager = ([host(t).copy() for t in ln], [host(t).copy() for t in acc], [host(w).copy() for w in work])
    for w, u in zip(work, Ups):
        w.copy_(u)
    api.dd_graph_begin(hs[0])
    try:
        api.dd_block_filter_batch(hs, Us, work, 3, n, 11, 5, ln, acc)
    finally:
        g = api.dd_graph_end(hs[0])
    # nothing ran during the capture
    assert all(np.array_equal(host(w), host(u)) for w, u in zip(work, Ups))
    for t in ln:
        t.zero_()
    api.dd_graph_launch(g, 0)
    got = ([host(t) for t in ln], [host(t) for t in acc], [host(w) for w in work])
    for a, b in zip(got, eager):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert api.dd_status(hs[0])[0] == 0
    api.dd_graph_destroy(g)
