"""Pins of the relative gauge fixing (Sec. 4) against the mathematics: the
functional never decreases, a proposal that is a pure gauge transform of U
is brought back to U, and determinant ratios and the plaquette are
unchanged by the fixing (gauge invariance)."""
import numpy as np

from oracle import dirac, estimator, gaugefix, geometry, heatbath
from paper_1112_1243_gb300 import synthetic


def test_functional_increases_and_recovers_pure_gauge():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.5, 21)
    h = synthetic.random_gauge_transform(dims, 22, eps=0.4)
    Up = dirac.gauge_transform_links(U, h, lat)
    g, Ug, hist = gaugefix.relative_gauge_fix(U, Up, lat, 60)
    assert all(b >= a - 1e-9 for a, b in zip(hist, hist[1:]))
    assert hist[-1] <= 12.0 * lat.V + 1e-9          # Re tr(1) = 3 on each of the 4V links
    assert np.max(np.abs(Ug - U)) < 1e-6
    # g is h^{-1} up to a global centre element: g h = c 1
    gh = g @ h
    c = gh[0, 0, 0]
    assert abs(abs(c) - 1) < 1e-6 and np.max(np.abs(gh - c * np.eye(3))) < 1e-6


def test_gauge_invariance_of_ratios_and_plaquette():
    dims, block, kappa = (4, 4, 4, 4), (2, 2, 2, 2), 0.12
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.4, 23)
    Up, _ = heatbath.gauge_update(U, lat, 5.3, 1, 0, 3, 1, colour_mask=3)
    g, Ug, hist = gaugefix.relative_gauge_fix(U, Up, lat, 5)
    assert hist[-1] > hist[0]
    ex = estimator.exact_ln_ratio_schur(U, Up, lat, kappa)
    exg = estimator.exact_ln_ratio_schur(U, Ug, lat, kappa)
    assert abs(ex - exg) < 1e-9 * max(1.0, abs(ex))
    for b in range(lat.nblocks):
        a1 = dirac.logabsdet(dirac.dense_dirichlet_block(Up, lat, kappa, b))
        a2 = dirac.logabsdet(dirac.dense_dirichlet_block(Ug, lat, kappa, b))
        assert abs(a1 - a2) < 1e-10
    assert abs(heatbath.plaquette_mean(Up, lat) - heatbath.plaquette_mean(Ug, lat)) < 1e-13
    # the fixed proposal differs from U on more links than the active ones
    assert gaugefix.differing_links(U, Ug).sum() > lat.active.sum()
