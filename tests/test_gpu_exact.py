"""GPU parity of the exact check path (dense LU) and of the exact block filter.

Tolerance: ln|det| of matrices up to 3072 x 3072 agree with LAPACK (numpy
slogdet of the oracle's independently built dense matrices) to 1e-9
relative: both are backward-stable LU factorisations with partial pivoting,
whose pivot orders may differ, so only rounding (~n * 1e-16 * cond) separates
them.
"""
import itertools

import numpy as np
import pytest

from oracle import accept, dirac, estimator, geometry, heatbath
from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api

pytestmark = pytest.mark.gpu
KAPPA = 0.12


@pytest.fixture(scope="module")
def api():
    return lib_api()


@pytest.fixture(scope="module")
def case():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.4, 1)
    return dims, block, lat, U


def test_logdet_full_and_free_field(api, case):
    dims, block, lat, U = case
    h = api.dd_init(dims, block, KAPPA)
    got = float(host(api.dd_logdet_exact(h, dev(U), 0))[0])
    ref = dirac.logabsdet(dirac.dense_D(U, lat, KAPPA))
    assert abs(got - ref) < 1e-9 * abs(ref)
    # free field: closed form 6 sum_p ln(a^2 + 4 k^2 sum sin^2 p)
    got0 = float(host(api.dd_logdet_exact(h, dev(synthetic.unit_gauge(dims)), 0))[0])
    cf = 0.0
    for n in itertools.product(*[range(L) for L in dims]):
        p = np.array([2 * np.pi * n[a] / dims[a] for a in range(3)] + [(2 * n[3] + 1) * np.pi / dims[3]])
        cf += 6 * np.log((1 - 2 * KAPPA * np.cos(p).sum()) ** 2 + 4 * KAPPA ** 2 * np.sum(np.sin(p) ** 2))
    assert abs(got0 - cf) < 1e-9 * abs(cf)


def test_logdet_blocks_and_schur(api, case):
    dims, block, lat, U = case
    h = api.dd_init(dims, block, KAPPA)
    gb = host(api.dd_logdet_exact(h, dev(U), 1))
    for b in range(lat.nblocks):
        ref = dirac.logabsdet(dirac.dense_dirichlet_block(U, lat, KAPPA, b))
        assert abs(gb[b] - ref) < 1e-10 * max(1.0, abs(ref))
    gs = float(host(api.dd_logdet_exact(h, dev(U), 2))[0])
    D = dirac.dense_D(U, lat, KAPPA)
    ref = dirac.logabsdet(dirac.dense_schur(D, lat))
    assert abs(gs - ref) < 1e-9 * max(1.0, abs(ref))
    # Eq. ddfactor on the GPU numbers alone
    gd = float(host(api.dd_logdet_exact(h, dev(U), 0))[0])
    assert abs(gd - (gb.sum() + gs)) < 1e-9 * abs(gd)


@pytest.mark.parametrize("cm", [1, 2])
def test_block_filter_exact(api, case, cm):
    dims, block, lat, U = case
    h = api.dd_init(dims, block, KAPPA)
    Up, _ = heatbath.gauge_update(U, lat, 5.3, 1, 0, 21, 4, colour_mask=cm)
    Upd = dev(Up)
    ln_b, acc = api.dd_block_filter(h, dev(U), Upd, cm, api.DD_FILTER_EXACT, 1, 33, 6)
    ref = estimator.block_ln_ratios_exact(U, Up, lat, KAPPA, colour_mask=cm)
    got = host(ln_b)
    assert np.max(np.abs(got - ref)) < 1e-9
    racc, lu = accept.block_accept(ref, 33, 6, cm, lat.block_colour)
    clear = np.abs(lu - ref) > 1e-8
    gacc = host(acc).astype(bool)
    assert np.array_equal(gacc[clear], racc[clear])
    assert np.array_equal(host(Upd), accept.restore_rejected_blocks(Up, U, lat, gacc))


def test_logdet_largest_panels(api):
    """The largest matrices of the exact path: on an 8 x 4^3 lattice (512
    sites) with 2 x 2^3 blocks, D is 6144 x 6144 and Dhat 3072 x 3072 (panels
    split over the thread blocks of one cooperative launch), the 16 block
    operators are 384 x 384 (one thread block per panel at the largest
    shared-memory panel), and the Schur assembly solves augmented 384 x 3456
    systems.  Against LAPACK on the oracle's matrices, and Eq. ddfactor."""
    dims, block = (8, 4, 4, 4), (4, 2, 2, 2)
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.4, 3)
    h = api.dd_init(dims, block, KAPPA)
    D = dirac.dense_D(U, lat, KAPPA)
    gd = float(host(api.dd_logdet_exact(h, dev(U), 0))[0])
    ref = dirac.logabsdet(D)
    assert abs(gd - ref) < 1e-9 * abs(ref)
    gb = host(api.dd_logdet_exact(h, dev(U), 1))
    for b in range(lat.nblocks):
        rb = dirac.logabsdet(dirac.dense_dirichlet_block(U, lat, KAPPA, b))
        assert abs(gb[b] - rb) < 1e-10 * max(1.0, abs(rb))
    gs = float(host(api.dd_logdet_exact(h, dev(U), 2))[0])
    rs = dirac.logabsdet(dirac.dense_schur(D, lat))
    assert abs(gs - rs) < 1e-9 * max(1.0, abs(rs))
    assert abs(gd - (gb.sum() + gs)) < 1e-9 * abs(gd)
    assert api.dd_status(h)[0] == 0


def test_tensor_core_update_matches_fp64_update(api, case):
    """The trailing update of the blocked LU on the tensor cores (Ozaki
    slices) against the FP64 FMA update: ln|det D| (3072^2) and ln|det Dhat|
    (1536^2) agree to FP64 rounding, both within 1e-9 of LAPACK."""
    dims, block, lat, U = case
    h = api.dd_init(dims, block, KAPPA)
    Ud = dev(U)
    got = {}
    for on in (True, False):
        api.dd_lu_tensor_cores(h, on)
        got[on] = (float(host(api.dd_logdet_exact(h, Ud, 0))[0]), float(host(api.dd_logdet_exact(h, Ud, 2))[0]))
    D = dirac.dense_D(U, lat, KAPPA)
    ref = (dirac.logabsdet(D), dirac.logabsdet(dirac.dense_schur(D, lat)))
    for k in range(2):
        assert abs(got[True][k] - got[False][k]) < 1e-11 * abs(ref[k]), (k, got[True][k], got[False][k])
        assert abs(got[True][k] - ref[k]) < 1e-9 * abs(ref[k])
    assert api.dd_status(h)[0] == 0
