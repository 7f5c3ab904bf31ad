"""Edge cases and degenerate inputs through the C ABI: rejected geometries
and arguments, an empty active set, a proposal equal to the current field
(every log-ratio vanishes), one right-hand side at the largest batch size,
and a lattice whose blocks are not cubes."""
import numpy as np
import pytest

from oracle import dirac, estimator, geometry
from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return lib_api()


@pytest.mark.parametrize("dims,block", [((5, 4, 4, 4), (1, 2, 2, 2)),     # odd extent
                                        ((8, 8, 8, 8), (3, 4, 4, 4)),     # block does not divide
                                        ((8, 8, 8, 8), (8, 4, 4, 4)),     # one block along axis 0
                                        ((12, 4, 4, 4), (4, 2, 2, 2))])   # three blocks along axis 0
def test_invalid_geometry_rejected(api, dims, block):
    with pytest.raises(api.DDError):
        api.dd_init(dims, block, 0.12)


def test_invalid_arguments_rejected(api):
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    h = api.dd_init(dims, block, 0.12, max_rhs=2)
    U = dev(synthetic.random_gauge(dims, 0.3, 1))
    with pytest.raises(api.DDError):
        api.dd_det_ratio_estimate(h, U, U, 3, 1, 1)          # n > max_rhs
    with pytest.raises(api.DDError):
        api.dd_block_filter(h, U, U.clone(), 0, api.DD_FILTER_STOCHASTIC, 1, 1, 1)   # empty colour mask
    with pytest.raises(api.DDError):
        api.dd_gauge_update(h, U, 3, -1.0, 1, 0, 1, 1)        # beta <= 0
    with pytest.raises(api.DDError):
        api.dd_block_schur_filter(h, U, U.clone(), 3, 1, 1, 1)  # no sub-blocks
    assert api.dd_status(h)[0] == 0


def test_empty_active_set(api):
    """2^4 blocks with the literal rule: every site is a boundary site, so
    nothing is active; the proposal and the filter change nothing."""
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    h = api.dd_init(dims, block, 0.12, active_mode=api.DD_ACTIVE_PAPER, max_rhs=2)
    assert not api.dd_get_maps(h)["active"].any()
    U = synthetic.random_gauge(dims, 0.3, 2)
    Ud = dev(U)
    api.dd_gauge_update(h, Ud, 3, 5.3, 2, 1, 3, 4)
    assert np.array_equal(host(Ud), U)
    Un = Ud.clone()
    ln_b, acc = api.dd_block_filter(h, Ud, Un, 3, api.DD_FILTER_STOCHASTIC, 2, 5, 6)
    assert np.all(host(ln_b) == 0.0)
    assert np.all(host(acc) == 1)
    assert api.dd_status(h)[0] == 0


def test_unchanged_proposal_gives_vanishing_ratios(api):
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.13
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.3, 7)
    h = api.dd_init(dims, block, kappa, max_rhs=3)
    Ud = dev(U)
    ln = host(api.dd_det_ratio_estimate(h, Ud, Ud, 3, 8, 9))
    # s = v - A a with a = A^{-1} v solved to tol_block: |ln r| <= 2 |eta| |D^{-1}| 1e-12 |v| (|v| <= |eta|)
    for i in range(3):
        eta = estimator.global_noise(lat, i, 8, 9)
        assert abs(ln[i]) <= 2 * np.linalg.norm(eta) ** 2 * 30 * 1e-12 * 10, (i, ln[i])
    for masked in (0, 1):
        api.dd_set_tuning(h, filter_masked=masked)
        ln_b, acc = api.dd_block_filter(h, Ud, Ud.clone(), 3, api.DD_FILTER_STOCHASTIC, 2, 1, 2)
        assert np.all(host(ln_b) == 0.0), masked
        assert np.all(host(acc) == 1)


def test_largest_batch_and_single_rhs_agree(api):
    """The same right-hand side solved alone and as the last of max_rhs
    right-hand sides gives the same solution to the solver tolerance."""
    dims, block, kappa = (8, 8, 8, 4), (4, 4, 4, 2), 0.12
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.3, 11)
    R = 6
    b = synthetic.random_spinor(dims, 12, nrhs=R)
    h = api.dd_init(dims, block, kappa, max_rhs=R, krylov=api.DD_KRYLOV_BICGSTAB)
    xs = dev(np.zeros_like(b))
    api.dd_solve(h, xs, dev(b), dev(U), R, api.DD_PREC_F16)
    x1 = dev(np.zeros_like(b[-1:]))
    api.dd_solve(h, x1, dev(b[-1:]), dev(U), 1, api.DD_PREC_F16)
    assert rel_err(host(xs)[-1], host(x1)[0]) < 1e-7
    true = np.linalg.norm(b[-1] - dirac.apply_D(U, host(xs)[-1], lat, kappa)) / np.linalg.norm(b[-1])
    assert true <= 1e-10 * 1.01


def test_non_cubic_blocks_dslash(api):
    dims, block, kappa = (12, 8, 4, 6), (6, 2, 2, 3), 0.11
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.5, 13)
    psi = synthetic.random_spinor(dims, 14)
    h = api.dd_init(dims, block, kappa)
    out = dev(np.zeros_like(psi))
    api.dd_apply_D(h, out, dev(psi), dev(U), api.DD_OP_D, api.DD_PREC_F64, 1)
    ref = dirac.apply_D(U, psi, lat, kappa)
    assert np.max(np.abs(host(out) - ref)) < 1e-13 * np.max(np.abs(ref))
    api.dd_apply_D_block(h, out, dev(psi), dev(U), 3, api.DD_PREC_F64, 1)
    assert rel_err(host(out), dirac.apply_D_dirichlet(U, psi, lat, kappa)) < 1e-12
