"""One level of recursive decomposition on the GPU (Eq. ddrec; Eq. 4step
steps 1 and 2) against the oracle: the sub-block filter (step 1) and the
blocks' Schur filter (step 2) with the same random streams; the recursive
chain step replayed as a CUDA graph against its eager run."""
import numpy as np
import pytest

from oracle import estimator, recursive
from oracle.interp import interpolate
from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api

pytestmark = pytest.mark.gpu

DIMS, BLOCK, SUB, KAPPA = (8, 8, 8, 8), (4, 4, 4, 4), (2, 2, 2, 2), 0.12


@pytest.fixture(scope="module")
def api():
    return lib_api()


@pytest.fixture(scope="module")
def tl():
    return recursive.TwoLevel(DIMS, BLOCK, SUB)


def perturbed(U, tl, eps, seed):
    R = synthetic.random_gauge(DIMS, eps, seed)
    Up = np.array(U, copy=True)
    Up[tl.active] = R[tl.active] @ U[tl.active]
    return Up


def test_maps_use_sub_block_active_links(api, tl):
    h = api.dd_init(DIMS, BLOCK, KAPPA, sub_block=SUB)
    maps = api.dd_get_maps(h)
    act = maps["active"] if isinstance(maps, dict) else maps[-1]
    assert np.array_equal(np.asarray(act).reshape(-1, 4).astype(bool), tl.active)
    with pytest.raises(api.DDError):
        api.dd_init(DIMS, BLOCK, KAPPA, sub_block=(4, 2, 2, 2))  # one sub-block along axis 0


@pytest.mark.parametrize("colour_mask", [3, 1])
def test_block_schur_filter_matches_oracle(api, tl, colour_mask):
    n, seed, ctr = 2, 41, 6
    U = synthetic.random_gauge(DIMS, 0.4, 51)
    Up = perturbed(U, tl, 0.25, 52)
    h = api.dd_init(DIMS, BLOCK, KAPPA, max_rhs=n, inner_prec=api.DD_PREC_F16, krylov=api.DD_KRYLOV_BICGSTAB,
                    sub_block=SUB)
    Un = dev(Up)
    ln_b, acc = api.dd_block_schur_filter(h, dev(U), Un, colour_mask, n, seed, ctr)
    got = host(ln_b)
    ref = recursive.block_schur_ln_ratios(U, Up, tl, KAPPA, n, seed, ctr, colour_mask=colour_mask, tol=1e-13)
    # block Dirichlet solve at 1e-10 relative: |d ln| <= 20 |eta| |D1'^{-1}|^2 1e-10 |eta| (|D1'^{-1}| < 10 here)
    for b in range(tl.lat1.nblocks):
        eta = recursive.block_schur_noise(tl, 0, seed, ctr, colour_mask)
        sel = tl.lat1.block_id == b
        bound = max(1e-8, n * 20 * np.linalg.norm(eta[sel]) ** 2 * 100 * 1e-10)
        assert abs(got[b] - ref[b]) <= bound, (b, got[b], ref[b], bound)
    # decisions and restore
    u_ln = np.log(np.array([float(x) for x in _uniforms(tl.lat1.nblocks, seed, ctr)]))
    a = host(acc).astype(bool)
    for b in range(tl.lat1.nblocks):
        if not (colour_mask >> int(tl.lat1.block_colour[b]) & 1):
            assert a[b]
        elif abs(u_ln[b] - ref[b]) > 1e-6:
            assert a[b] == (u_ln[b] < ref[b])
    out = host(Un)
    rej = ~a[tl.lat1.block_id]
    m = tl.active & rej[:, None]
    assert np.array_equal(out[m], U[m])
    assert np.array_equal(out[~m], Up[~m])
    assert api.dd_status(h)[0] == 0


def _uniforms(nb, seed, ctr):
    from oracle import rng
    return rng.accept_uniform(np.arange(nb, dtype=np.uint64), recursive.PURPOSE_BLOCK_SCHUR_ACCEPT, seed, ctr)


def test_sub_block_filter_matches_oracle(api, tl):
    """dd_block_filter on a handle with sub-blocks filters the sub-blocks
    (step 1), colour by colour as the intra-block active set requires."""
    n, seed, ctr = 2, 43, 7
    U = synthetic.random_gauge(DIMS, 0.4, 53)
    Up = perturbed(U, tl, 0.25, 54)
    h = api.dd_init(DIMS, BLOCK, KAPPA, max_rhs=n, sub_block=SUB)
    lat2 = tl.lat2
    only_black = np.array(U, copy=True)
    m = tl.active & (lat2.colour == 0)[:, None]
    only_black[m] = Up[m]
    ln_b, acc = api.dd_block_filter(h, dev(U), dev(only_black), 1, api.DD_FILTER_STOCHASTIC, n, seed, ctr)
    got = host(ln_b)
    assert got.shape == (lat2.nblocks,)
    ref = estimator.block_ln_ratios(U, only_black, lat2, KAPPA, n, seed, ctr, colour_mask=1, tol=1e-14)
    assert np.max(np.abs(got - ref)) < 1e-8 * max(1.0, np.max(np.abs(ref)))


def test_recursive_chain_graph_equals_eager(api):
    """16^4 lattice, 8^4 blocks, 4^4 sub-blocks (96 active links per
    sub-block): steps 0-3 with the blocks' Schur filter, eager against a
    graph replay, bit for bit."""
    from paper_1112_1243_gb300.chain import HierarchicalStep
    dims, block, sub = (16, 16, 16, 16), (8, 8, 8, 8), (4, 4, 4, 4)
    U = synthetic.random_gauge(dims, 0.25, 61)

    def mk():
        h = api.dd_init(dims, block, 0.13, max_rhs=2, inner_prec=api.DD_PREC_F16, krylov=api.DD_KRYLOV_BICGSTAB,
                        sub_block=sub)
        return h, HierarchicalStep(h, 5.3, n_inner=1, n_block=2, n_global=2, seed=5, n_schur=2)

    ha, ca = mk()
    Ua = dev(U)
    eager = []
    for k in range(2):
        ln, acc = ca.step(Ua, k)
        eager.append((host(ln).copy(), host(ca.ln_b).copy(), host(ca.ln_bs).copy(), host(Ua).copy()))
        assert np.all(np.isfinite(eager[-1][2]))
    assert api.dd_status(ha)[0] == 0
    hb, cb = mk()
    Ub = dev(U)
    cb.capture(Ub)
    for k in range(2):
        cb.step_graph(k)
        got = (host(cb.ln_g), host(cb.ln_b), host(cb.ln_bs), host(Ub))
        for x, y in zip(got, eager[k]):
            assert np.array_equal(x, y), k
    assert api.dd_status(hb)[0] == 0
