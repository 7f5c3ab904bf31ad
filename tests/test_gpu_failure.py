"""Failure paths of the library, driven by host-made inputs (nothing here
faults a GPU): an iteration cap the solver cannot meet, a gauge field with a
non-finite entry, and a grid barrier that waits for an arrival that never
comes.  Every call returns its documented error code, and the device status
word (read and cleared by dd_status) carries the same code where the work
ran without host polling (a replayed CUDA graph).  The only kernel of the
library that waits on other thread blocks is the cooperative LU panel
launch; its barrier gives up after a bounded number of polls."""
import time

import numpy as np
import pytest

from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api

pytestmark = pytest.mark.gpu

DIMS, BLOCK, KAPPA = (8, 8, 8, 8), (4, 4, 4, 4), 0.13


@pytest.fixture(scope="module")
def api():
    return lib_api()


def solver_cases(api):
    return [(api.DD_PREC_F64, api.DD_KRYLOV_CGNR), (api.DD_PREC_F16, api.DD_KRYLOV_BICGSTAB),
            (api.DD_PREC_F16, api.DD_KRYLOV_CGNR)]


def test_iteration_cap_reports_not_converged(api):
    import torch
    U = dev(synthetic.random_gauge(DIMS, 0.3, 5))
    b = dev(synthetic.random_spinor(DIMS, 6))
    for prec, krylov in solver_cases(api):
        h = api.dd_init(DIMS, BLOCK, KAPPA, max_rhs=1, inner_prec=prec, krylov=krylov, maxit=1)
        x = torch.zeros_like(b)
        it, res, rc = api.dd_solve(h, x, b, U, 1, prec, check=False)
        assert rc == api.DD_ERR_NOT_CONVERGED, (prec, krylov, rc)
        assert res[0] > 1e-10 and np.isfinite(res[0])
        assert "maxit" in api.dd_last_error(h) or "cap" in api.dd_last_error(h)
        assert api.dd_status(h)[0] == 0              # eager: reported by the return code
        # the same solve recorded as a CUDA graph: no host polling, the
        # device status word reports the missed target
        api.dd_graph_begin(h)
        try:
            api.dd_solve(h, x, b, U, 1, prec, check=False)
        finally:
            g = api.dd_graph_end(h)
        api.dd_graph_launch(g, 0)
        assert api.dd_status(h)[0] == api.DD_ERR_NOT_CONVERGED, (prec, krylov)
        assert api.dd_status(h)[0] == 0              # read and cleared
        api.dd_graph_destroy(g)
        # with a reachable cap the handle works again
        h2 = api.dd_init(DIMS, BLOCK, KAPPA, max_rhs=1, inner_prec=prec, krylov=krylov)
        it, res, rc = api.dd_solve(h2, x, b, U, 1, prec, check=False)
        assert rc == api.DD_OK and res[0] <= 1e-10


def poisoned_field():
    """A gauge field with one NaN entry, on a link inside a white block
    (site x = (5, 1, 1, 1): block coordinates (1, 0, 0, 0))."""
    U = synthetic.random_gauge(DIMS, 0.3, 7)
    s = 5 + 8 * (1 + 8 * (1 + 8 * 1))
    U[s, 1, 0, 0] = complex(np.nan, 0.0)
    return U


def test_non_finite_gauge_field_reports_numeric(api):
    import torch
    Un = dev(poisoned_field())
    b = dev(synthetic.random_spinor(DIMS, 8))
    for prec, krylov in solver_cases(api):
        h = api.dd_init(DIMS, BLOCK, KAPPA, max_rhs=1, inner_prec=prec, krylov=krylov)
        x = torch.zeros_like(b)
        it, res, rc = api.dd_solve(h, x, b, Un, 1, prec, check=False)
        assert rc == api.DD_ERR_NUMERIC, (prec, krylov, rc)
        assert api.dd_status(h)[0] == api.DD_ERR_NUMERIC
    # the global stochastic estimate (Schur pieces and global solve) on it
    h = api.dd_init(DIMS, BLOCK, KAPPA, max_rhs=2, inner_prec=api.DD_PREC_F16, krylov=api.DD_KRYLOV_BICGSTAB)
    with pytest.raises(api.DDError) as e:
        api.dd_det_ratio_estimate(h, Un, Un.clone(), 2, 5, 3)
    assert e.value.code == api.DD_ERR_NUMERIC
    assert api.dd_status(h)[0] == api.DD_ERR_NUMERIC
    # a finite field on the same handle afterwards: no error
    U = dev(synthetic.random_gauge(DIMS, 0.3, 7))
    Up = U.clone()
    api.dd_gauge_update(h, Up, 3, 5.3, 1, 0, 11, 3)
    ln = api.dd_det_ratio_estimate(h, U, Up, 2, 5, 3)
    assert np.all(np.isfinite(host(ln)))
    assert api.dd_status(h)[0] == 0


def test_grid_barrier_wait_is_bounded(api):
    """The grid barrier of the LU panel launch: all arrivals -> passed, no
    status; one arrival missing -> the wait gives up within seconds, the
    status word reads DD_ERR_TIMEOUT, and the context still works (an exact
    determinant right after matches the one before)."""
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    h = api.dd_init(dims, block, 0.12)
    U = dev(synthetic.random_gauge(dims, 0.4, 1))
    ref = float(host(api.dd_logdet_exact(h, U, 0))[0])
    assert api.dd_barrier_check(h, 0) is True
    assert api.dd_status(h)[0] == 0
    t0 = time.time()
    assert api.dd_barrier_check(h, 1) is False
    waited = time.time() - t0
    assert api.dd_status(h)[0] == api.DD_ERR_TIMEOUT
    assert waited < 60.0
    assert api.dd_status(h)[0] == 0              # read and cleared
    assert float(host(api.dd_logdet_exact(h, U, 0))[0]) == ref
    assert api.dd_status(h)[0] == 0
