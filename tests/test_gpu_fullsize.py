"""Parity at the full benchmark size: the 32^3 x 64 lattice with 8^4 blocks,
kappa 0.1355 and the eps = 0.2 synthetic field the benchmark uses (seed 5),
in the launch configuration the benchmark times (12 right-hand sides per
batched launch).  The oracle applies D on the whole lattice (a few seconds
of numpy per application), so:
  * Dslash (FP64 and the FP16-storage path) is compared on every site;
  * the mixed-precision solve is checked through the oracle's own true
    residual ||b - D x|| / ||b|| of the GPU solution (a property that holds
    at any size);
  * the Dirichlet block operator of both colours is compared on every site.
"""
import numpy as np
import pytest

from oracle import dirac, geometry
from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DIMS, BLOCK, KAPPA, EPS, SEED = (32, 32, 32, 64), (8, 8, 8, 8), 0.1355, 0.2, 5


@pytest.fixture(scope="module")
def api():
    return lib_api()


@pytest.fixture(scope="module")
def setup(api):
    lat = geometry.Lattice(DIMS, BLOCK)
    U = synthetic.random_gauge(DIMS, EPS, SEED)
    return lat, U


def test_dslash_fullsize(api, setup):
    lat, U = setup
    h = api.dd_init(DIMS, BLOCK, KAPPA, max_rhs=1, features=api.DD_FEAT_SOLVE)
    psi = synthetic.random_spinor(DIMS, 21)
    ref = dirac.apply_D(U, psi, lat, KAPPA)
    Ud, pd = dev(U), dev(psi)
    out = dev(np.zeros_like(psi))
    api.dd_apply_D(h, out, pd, Ud, api.DD_OP_D, api.DD_PREC_F64, 1)
    got = host(out)
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))
    api.dd_apply_D(h, out, pd, Ud, api.DD_OP_D, api.DD_PREC_F16, 1)
    assert rel_err(host(out), ref) < 2e-3
    # Dirichlet operator of each colour
    refb = dirac.apply_D_dirichlet(U, psi, lat, KAPPA)
    for cm in (1, 2):
        api.dd_apply_D_block(h, out, pd, Ud, cm, api.DD_PREC_F64, 1)
        sel = lat.colour == (0 if cm == 1 else 1)
        got = host(out)
        assert np.max(np.abs(got[sel] - refb[sel])) < 1e-13 * np.max(np.abs(refb))
        assert not np.any(got[~sel])


def test_mixed_solve_fullsize_true_residual(api, setup):
    """Two right-hand sides in one batched mixed FP16/FP32 + FP64 solve (the
    benchmark's global-solve configuration, BiCGStab inner solver)."""
    lat, U = setup
    nrhs = 2
    h = api.dd_init(DIMS, BLOCK, KAPPA, max_rhs=nrhs, features=api.DD_FEAT_SOLVE, tol_global=1e-10,
                    krylov=api.DD_KRYLOV_BICGSTAB, maxit=40000)
    b = synthetic.random_spinor(DIMS, 22, nrhs=nrhs)
    x = dev(np.zeros_like(b))
    it, res, rc = api.dd_solve(h, x, dev(b), dev(U), nrhs, api.DD_PREC_F16)
    xh = host(x)
    for r in range(nrhs):
        true = np.linalg.norm(b[r] - dirac.apply_D(U, xh[r], lat, KAPPA)) / np.linalg.norm(b[r])
        assert true <= 1e-10 * 1.01, (r, true, res)
        assert abs(true - res[r]) <= 1e-11 + 0.1 * true
