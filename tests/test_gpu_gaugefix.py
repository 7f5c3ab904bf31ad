"""Relative gauge fixing (Sec. 4) on the GPU against the oracle: the fixed
field element by element, the recovery of a pure gauge transform, the
global estimate of the fixed proposal (interpolation over every differing
link) and the chain step with fixing."""
import numpy as np
import pytest

from oracle import chain, dirac, estimator, gaugefix, geometry, heatbath
from oracle.interp import interpolate
from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return lib_api()


def test_fixed_field_matches_oracle(api):
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.4, 71)
    Up, _ = heatbath.gauge_update(U, lat, 5.3, 1, 0, 72, 1)
    g, Ug, hist = gaugefix.relative_gauge_fix(U, Up, lat, 4)
    h = api.dd_init(dims, block, 0.13)
    Upd = dev(Up)
    import torch
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    api.dd_relative_gauge_fix(h, dev(U), Upd, 4, F)
    assert np.max(np.abs(host(Upd) - Ug)) < 1e-12
    assert abs(float(host(F)[0]) - hist[-1]) < 1e-9 * abs(hist[-1])
    assert hist[-1] > hist[0]


def test_recovers_pure_gauge_transform(api):
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.5, 73)
    gt = synthetic.random_gauge_transform(dims, 74, eps=0.4)
    Up = dirac.gauge_transform_links(U, gt, lat)
    h = api.dd_init(dims, block, 0.12)
    Upd = dev(Up)
    api.dd_relative_gauge_fix(h, dev(U), Upd, 60)
    assert np.max(np.abs(host(Upd) - U)) < 1e-6


def test_estimate_of_fixed_proposal(api):
    dims, block, kappa, n = (4, 4, 4, 4), (2, 2, 2, 2), 0.12, 2
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.4, 75)
    Up, _ = heatbath.gauge_update(U, lat, 5.3, 1, 0, 76, 1, colour_mask=3)
    _, Ug, _ = gaugefix.relative_gauge_fix(U, Up, lat, 3)
    h = api.dd_init(dims, block, kappa, max_rhs=n, inner_prec=api.DD_PREC_F64)
    got = host(api.dd_det_ratio_estimate(h, dev(U), dev(Ug), n, 5, 3,
                                         api.DD_EST_FACTORS | api.DD_EST_INTERP_ALL))
    mask = gaugefix.differing_links(U, Ug)
    ref = estimator.det_ratio_estimate(U, Ug, lat, kappa, n, 5, 3, tol=1e-14, interp_mask=mask)
    D = dirac.dense_D(Ug, lat, kappa)
    dn = 1.0 / np.linalg.svd(D, compute_uv=False)[-1]
    for i in range(n):
        eta = estimator.global_noise(lat, i, 5, 3)
        Ui = interpolate(U, Ug, i / n, mask)
        Uj = interpolate(U, Ug, (i + 1) / n, mask)
        s = estimator.delta_source(Ui, Uj, eta, lat, kappa)
        d = np.linalg.norm(s) * dn
        bound = max(1e-8, 20 * (np.linalg.norm(eta) + d) * dn * 1e-10 * np.linalg.norm(s))
        assert abs(got[i] - ref[i]) <= bound, (i, got[i], ref[i], bound)


def test_chain_step_with_gauge_fixing(api):
    from paper_1112_1243_gb300.chain import HierarchicalStep
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.13
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.3, 77)
    h = api.dd_init(dims, block, kappa, max_rhs=2, inner_prec=api.DD_PREC_F16)
    st = HierarchicalStep(h, 5.3, n_inner=1, n_block=2, n_global=2, seed=4321, gauge_fix_sweeps=3)
    Ud = dev(U)
    Uo = U.copy()
    for k in range(2):
        ln_g, acc = st.step(Ud, k)
        Uo, rec = chain.hierarchical_step(Uo, lat, kappa, 5.3, 1, 2, 2, 4321, k, gauge_fix_sweeps=3)
        assert np.max(np.abs(host(ln_g) - rec["ln_global"])) < 1e-6
        margin = abs(float(np.sum(rec["ln_global"])) - rec["ln_u"])
        assert margin > 1e-6, "near tie: not compared"
        assert bool(host(acc)[0]) == rec["accept"]
        assert np.max(np.abs(host(Ud) - Uo)) < 1e-10
    assert api.dd_status(h)[0] == 0
