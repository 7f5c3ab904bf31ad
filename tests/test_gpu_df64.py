"""Defect correction with the true residual in double-float arithmetic
(outer_prec = DD_PREC_DF64): the solves still meet the FP64 target on the
oracle's own operator, whole-lattice and Dirichlet (block-colour) solves
inside the estimator agree with the oracle, right-hand sides far outside
FP32's exponent range are handled by the per-system power-of-two scale, and
a captured graph replays the eager solve bit for bit."""
import numpy as np
import pytest

from oracle import dirac, estimator, geometry, heatbath
from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return lib_api()


@pytest.mark.parametrize("prec,krylov", [(1, 0), (2, 0), (1, 1), (2, 1)])
def test_solve_true_residual_df(api, prec, krylov):
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.13
    nrhs = 3
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.3, 2)
    b = synthetic.random_spinor(dims, 11, nrhs=nrhs)
    h = api.dd_init(dims, block, kappa, max_rhs=nrhs, tol_global=1e-10, krylov=krylov,
                    outer_prec=api.DD_PREC_DF64)
    x = dev(np.zeros_like(b))
    it, res, rc = api.dd_solve(h, x, dev(b), dev(U), nrhs, prec)
    xh = host(x)
    for r in range(nrhs):
        true = np.linalg.norm(b[r] - dirac.apply_D(U, xh[r], lat, kappa)) / np.linalg.norm(b[r])
        assert true <= 1e-10 * 1.01, (prec, r, true, res)
        # the reported residual is the double-float one: within 2^-40 |x| / |b| of the FP64 value
        assert abs(true - res[r]) <= 1e-12 + 0.01 * true
    # the same systems with the FP64 residual: solutions agree to the solver tolerance
    h64 = api.dd_init(dims, block, kappa, max_rhs=nrhs, tol_global=1e-10, krylov=krylov)
    x64 = dev(np.zeros_like(b))
    api.dd_solve(h64, x64, dev(b), dev(U), nrhs, prec)
    assert rel_err(xh, host(x64)) < 1e-8


@pytest.mark.parametrize("scale", [1e-40, 1e40])
def test_rhs_outside_fp32_range(api, scale):
    """|b| of 1e-40 or 1e40 (FP32 underflows / overflows): the power-of-two
    scale keeps the double-float vectors in range; x scales with b."""
    dims, block, kappa = (4, 4, 4, 8), (2, 2, 2, 4), 0.12
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.4, 21)
    b = synthetic.random_spinor(dims, 22)
    h = api.dd_init(dims, block, kappa, max_rhs=1, krylov=1, outer_prec=api.DD_PREC_DF64)
    x1 = dev(np.zeros_like(b))
    api.dd_solve(h, x1, dev(b), dev(U), 1, api.DD_PREC_F16)
    xs = dev(np.zeros_like(b))
    api.dd_solve(h, xs, dev(b * scale), dev(U), 1, api.DD_PREC_F16)
    xsh = host(xs)
    true = np.linalg.norm(b * scale - dirac.apply_D(U, xsh, lat, kappa)) / np.linalg.norm(b * scale)
    assert true <= 1e-10 * 1.01
    assert rel_err(xsh / scale, host(x1)) < 1e-8


@pytest.mark.parametrize("n", [1, 3])
def test_global_estimate_df(api, n):
    """Every solve of the estimate (global, and the Dirichlet solves of the
    Schur pieces over one block colour) with the double-float residual."""
    dims, block, kappa = (4, 4, 4, 4), (2, 2, 2, 2), 0.12
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.4, 1)
    Up, _ = heatbath.gauge_update(U, lat, 5.3, 1, 0, 77, 1, colour_mask=3)
    h = api.dd_init(dims, block, kappa, max_rhs=n, inner_prec=api.DD_PREC_F16, krylov=1,
                    outer_prec=api.DD_PREC_DF64)
    got = host(api.dd_det_ratio_estimate(h, dev(U), dev(Up), n, 5, 3, api.DD_EST_FACTORS))
    ref = estimator.det_ratio_estimate(U, Up, lat, kappa, n, 5, 3, tol=1e-14)
    D = dirac.dense_D(Up, lat, kappa)
    dn = 1.0 / np.linalg.svd(D, compute_uv=False)[-1]
    from oracle.interp import interpolate
    for i in range(n):
        eta = estimator.global_noise(lat, i, 5, 3)
        Ui = interpolate(U, Up, i / n, lat.active)
        Uj = interpolate(U, Up, (i + 1) / n, lat.active)
        s = estimator.delta_source(Ui, Uj, eta, lat, kappa)
        d = np.linalg.norm(s) * dn
        bound = max(1e-8, 20 * (np.linalg.norm(eta) + d) * dn * 1e-10 * np.linalg.norm(s))
        assert abs(got[i] - ref[i]) <= bound, (i, got[i], ref[i], bound)
    assert api.dd_status(h)[0] == 0


def test_chain_step_df(api):
    """Two hierarchical steps with the double-float residual: log-ratios and
    accept decisions as the oracle's chain."""
    from oracle import chain
    from paper_1112_1243_gb300.chain import HierarchicalStep
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.13
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.3, 77)
    h = api.dd_init(dims, block, kappa, max_rhs=2, inner_prec=api.DD_PREC_F16, krylov=1,
                    outer_prec=api.DD_PREC_DF64)
    st = HierarchicalStep(h, 5.3, n_inner=1, n_block=2, n_global=2, seed=4321)
    Ud = dev(U)
    Uo = U.copy()
    for k in range(2):
        ln_g, acc = st.step(Ud, k)
        Uo, rec = chain.hierarchical_step(Uo, lat, kappa, 5.3, 1, 2, 2, 4321, k)
        assert np.max(np.abs(host(ln_g) - rec["ln_global"])) < 1e-6
        margin = abs(float(np.sum(rec["ln_global"])) - rec["ln_u"])
        assert margin > 1e-6, "near tie: not compared"
        assert bool(host(acc)[0]) == rec["accept"]
        assert np.max(np.abs(host(Ud) - Uo)) < 1e-10
    assert api.dd_status(h)[0] == 0


def test_graph_of_df_solve_matches_eager(api):
    import torch
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    U = synthetic.random_gauge(dims, 0.3, 5)
    b = synthetic.random_spinor(dims, 6, nrhs=2)
    h = api.dd_init(dims, block, 0.13, max_rhs=2, inner_prec=api.DD_PREC_F16, krylov=1,
                    outer_prec=api.DD_PREC_DF64)
    Ud, bd = dev(U), dev(b)
    x_eager = torch.zeros_like(bd)
    api.dd_solve(h, x_eager, bd, Ud, nrhs=2, prec=api.DD_PREC_F16)
    x_graph = torch.zeros_like(bd)
    api.dd_graph_begin(h)
    try:
        api.dd_solve(h, x_graph, bd, Ud, nrhs=2, prec=api.DD_PREC_F16)
    finally:
        g = api.dd_graph_end(h)
    api.dd_graph_launch(g, 0)
    assert np.array_equal(host(x_graph), host(x_eager))
    assert api.dd_status(h)[0] == 0
    api.dd_graph_destroy(g)


def test_invalid_outer_prec_rejected(api):
    with pytest.raises(api.DDError):
        api.dd_init((4, 4, 4, 4), (2, 2, 2, 2), 0.12, outer_prec=api.DD_PREC_F32)
