"""Pins of the recursive-decomposition oracle (Eq. ddrec, Eq. 4step step 2)
against the mathematics: the factorisation det D_b = prod det D_b' det Dhat_b
by independent dense LU, the delta form against the dense definition of
-(|M_b eta|^2 - |eta|^2), the no-change case, and the decoupling of blocks."""
import numpy as np
import pytest

from oracle import dirac, recursive
from paper_1112_1243_gb300 import synthetic

DIMS, BLOCK, SUB = (8, 4, 4, 4), (4, 4, 4, 4), (2, 2, 2, 2)
KAPPA = 0.12


@pytest.fixture(scope="module")
def tl():
    return recursive.TwoLevel(DIMS, BLOCK, SUB)


def perturb_active(U, tl, eps, seed):
    """U' = U exp(i eps H) on the active links only (a generic proposal)."""
    R = synthetic.random_gauge(DIMS, eps, seed)
    Up = np.array(U, copy=True)
    m = tl.active
    Up[m] = R[m] @ U[m]
    return Up


def test_sub_blocks_must_tile_evenly():
    with pytest.raises(ValueError):
        recursive.TwoLevel((8, 8, 8, 8), (4, 4, 4, 4), (4, 2, 2, 2))   # one sub-block along axis 0
    with pytest.raises(ValueError):
        recursive.TwoLevel((12, 12, 12, 12), (6, 6, 6, 6), (2, 2, 2, 2))  # three per direction


def test_factorisation_of_block_determinants(tl):
    U = synthetic.random_gauge(DIMS, 0.5, 31)
    lat1, lat2 = tl.lat1, tl.lat2
    for blk in range(lat1.nblocks):
        lhs = dirac.logabsdet(dirac.dense_dirichlet_block(U, lat1, KAPPA, blk))
        sites = lat1.block_sites_of(blk)
        subs = np.unique(lat2.block_id[sites])
        assert len(subs) == 16
        rhs = sum(dirac.logabsdet(dirac.dense_dirichlet_block(U, lat2, KAPPA, int(b))) for b in subs)
        rhs += dirac.logabsdet(recursive.dense_block_schur(U, tl, KAPPA, blk))
        assert abs(lhs - rhs) < 1e-9 * max(1.0, abs(lhs))


def test_delta_form_equals_dense_definition(tl):
    U = synthetic.random_gauge(DIMS, 0.4, 32)
    Up = perturb_active(U, tl, 0.3, 33)
    n, seed, ctr = 1, 77, 5
    ln = recursive.block_schur_ln_ratios(U, Up, tl, KAPPA, n, seed, ctr)
    eta = recursive.block_schur_noise(tl, 0, seed, ctr)
    for blk in range(tl.lat1.nblocks):
        ref = recursive.block_schur_ln_factor_dense(U, Up, eta, tl, KAPPA, blk)
        assert abs(ln[blk] - ref) < 1e-8 * max(1.0, abs(ref)), (blk, ln[blk], ref)
    # the noise lives exactly on the black sub-blocks
    on = np.any(eta != 0, axis=(1, 2))
    assert np.array_equal(on, tl.lat2.colour == 0)


def test_no_change_gives_zero(tl):
    U = synthetic.random_gauge(DIMS, 0.4, 34)
    ln = recursive.block_schur_ln_ratios(U, U, tl, KAPPA, 2, 1, 2)
    # s = v - D_b a with a = A^{-1} v from a CG at 1e-14: zero to that accuracy
    assert np.max(np.abs(ln)) < 1e-11
    assert np.all(recursive.block_schur_ln_ratios_exact(U, U, tl, KAPPA) == 0.0)


def test_blocks_decouple(tl):
    """Changing the active links of one block changes only that block's
    Schur ratio (exact), and the ratio of the other block stays 0."""
    U = synthetic.random_gauge(DIMS, 0.4, 35)
    Up = perturb_active(U, tl, 0.3, 36)
    only0 = np.array(U, copy=True)
    m = tl.active & (tl.lat1.block_id == 0)[:, None]
    only0[m] = Up[m]
    ex = recursive.block_schur_ln_ratios_exact(U, only0, tl, KAPPA)
    assert ex[0] != 0.0 and ex[1] == 0.0
    full = recursive.block_schur_ln_ratios_exact(U, Up, tl, KAPPA)
    assert abs(full[0] - ex[0]) < 1e-10


def test_exact_ratios_telescope_through_the_hierarchy(tl):
    """Sum over blocks of the step-2 exact log-ratios plus the sub-block
    (step-1) exact log-ratios = 2 (ln|det D1'| - ln|det D1|) for the block
    Dirichlet operator (Eq. ddrec applied to both fields)."""
    from oracle import estimator
    U = synthetic.random_gauge(DIMS, 0.4, 37)
    Up = perturb_active(U, tl, 0.2, 38)
    lat1, lat2 = tl.lat1, tl.lat2
    s2 = recursive.block_schur_ln_ratios_exact(U, Up, tl, KAPPA).sum()
    s1 = estimator.block_ln_ratios_exact(U, Up, lat2, KAPPA).sum()
    d1 = sum(2.0 * (dirac.logabsdet(dirac.dense_dirichlet_block(Up, lat1, KAPPA, b))
                    - dirac.logabsdet(dirac.dense_dirichlet_block(U, lat1, KAPPA, b))) for b in range(lat1.nblocks))
    assert abs((s1 + s2) - d1) < 1e-8 * max(1.0, abs(d1))
