"""The Schwarz-preconditioned flexible GCR (krylov DD_KRYLOV_SAP_GCR) against
the oracle (oracle/schwarz.py):
  * the preconditioner alone (dd_sap_apply) with block solves of 64 FP32
    BiCGStab iterations reproduces the oracle's Schwarz cycles with exact
    (dense LU) block solves, to FP32 accuracy (relative 2e-5): same colour
    order, same residual of each colour's sites;
  * SAP-GCR solves meet the true residual 1e-10 of the oracle's own operator
    and agree with the BiCGStab solution within the conditioning of D.
"""
import numpy as np
import pytest

from oracle import dirac, geometry, schwarz
from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return lib_api()


@pytest.mark.parametrize("dims,block,kappa", [((4, 4, 4, 4), (2, 2, 2, 2), 0.12), ((8, 4, 4, 4), (4, 2, 2, 2), 0.12),
                                             ((8, 8, 8, 8), (4, 4, 4, 4), 0.13)])
@pytest.mark.parametrize("ncy", [1, 2])
def test_sap_apply_matches_oracle(api, dims, block, kappa, ncy):
    import torch
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.3, 51)
    rho = synthetic.random_spinor(dims, 52, nrhs=2)
    h = api.dd_init(dims, block, kappa, max_rhs=2, inner_prec=api.DD_PREC_F32, krylov=api.DD_KRYLOV_SAP_GCR,
                    sap_ncy=ncy, sap_nmr=64, sap_nkv=2)
    out = torch.zeros_like(dev(rho))
    api.dd_sap_apply(h, out, dev(rho), dev(U), 2, api.DD_PREC_F32)
    got = host(out)
    blocks = schwarz.BlockSolver(U, lat, kappa)
    for k in range(2):
        ref = schwarz.sap(U, lat, kappa, rho[k], ncy, blocks)
        assert rel_err(got[k], ref) < 2e-5, (k, rel_err(got[k], ref))
    assert api.dd_status(h)[0] == 0


@pytest.mark.parametrize("dims,block,kappa,prec", [((4, 4, 4, 4), (2, 2, 2, 2), 0.12, 2),
                                                  ((8, 8, 8, 8), (4, 4, 4, 4), 0.13, 2),
                                                  ((8, 8, 8, 8), (4, 4, 4, 4), 0.13, 1)])
def test_sap_gcr_solve_true_residual(api, dims, block, kappa, prec):
    import torch
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.3, 53)
    b = synthetic.random_spinor(dims, 54, nrhs=2)
    Ud, bd = dev(U), dev(b)
    h = api.dd_init(dims, block, kappa, max_rhs=2, inner_prec=prec, krylov=api.DD_KRYLOV_SAP_GCR)
    x = torch.zeros_like(bd)
    it, res, rc = api.dd_solve(h, x, bd, Ud, 2, prec)
    assert rc == api.DD_OK and max(res) <= 1e-10 and it > 0
    xs = host(x)
    hb = api.dd_init(dims, block, kappa, max_rhs=2, inner_prec=prec, krylov=api.DD_KRYLOV_BICGSTAB)
    xb = torch.zeros_like(bd)
    api.dd_solve(hb, xb, bd, Ud, 2, prec)
    xbh = host(xb)
    for k in range(2):
        true = np.linalg.norm(b[k] - dirac.apply_D(U, xs[k], lat, kappa)) / np.linalg.norm(b[k])
        assert true <= 1.01e-10, (k, true)
        assert rel_err(xs[k], xbh[k]) < 1e-8
    assert api.dd_status(h)[0] == 0
