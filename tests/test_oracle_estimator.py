"""Oracle pins for the stochastic estimator, interpolation, heat-bath and
acceptance law.

Pins: E[exp(-eta^dag (A - 1) eta)] = 1/det A and the variance
prod(2 lambda - 1)^{-1} - prod lambda^{-2} (Sec. 4), the closed-form geodesic
exp(i t eps H), the erfc acceptance law (Eq. acceptance), the rank bound on
eigenvalues of M^dag M equal to one (Sec. 4: the Schur complement acts on
boundary points only), the Kennedy-Pendleton density, action conservation of
over-relaxation and the strong-coupling plaquette beta/18 + beta^2/216.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import accept, dirac, estimator, geometry, heatbath, interp, rng
from paper_1112_1243_gb300 import synthetic

KAPPA = 0.12


# ----------------------------------------------------------------- estimator
def _small_hpd(dim, seed, lo=0.62, hi=1.6):
    rs = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rs.standard_normal((dim, dim)) + 1j * rs.standard_normal((dim, dim)))
    lam = rs.uniform(lo, hi, dim)
    return Q @ np.diag(lam) @ Q.conj().T, lam


def test_estimator_mean_and_variance():
    """Sec. 4: with p(eta) ~ exp(-eta^dag eta), E exp(-eta^dag(A-1)eta) = 1/det A;
    the variance prod(2l-1)^-1 - prod l^-2 exists for l > 1/2."""
    dim, n = 6, 400000
    # lambda > 3/4 keeps the fourth moment finite, so the sample variance converges
    A, lam = _small_hpd(dim, 1, lo=0.85, hi=1.5)
    el = np.arange(n * dim, dtype=np.uint64)
    eta = rng.gaussian_components(el, rng.PURPOSE_USER_NOISE, 0, 2024, 1).reshape(n, dim)
    q = np.einsum("ni,ij,nj->n", np.conj(eta), A - np.eye(dim), eta).real
    w = np.exp(-q)
    mean_ref = 1.0 / np.prod(lam)
    var_ref = 1.0 / np.prod(2 * lam - 1) - 1.0 / np.prod(lam) ** 2
    assert abs(w.mean() - mean_ref) < 5 * math.sqrt(var_ref / n)
    se_var = np.std((w - w.mean()) ** 2) / math.sqrt(n)
    assert abs(w.var() - var_ref) < 5 * se_var


def test_delta_form_equals_definition():
    """ln r_i through delta = (M - 1) eta equals -(|M eta|^2 - |eta|^2) with dense M."""
    dims = (4, 4, 4, 4)
    lat = geometry.Lattice(dims, (2, 2, 2, 2))
    U = synthetic.random_gauge(dims, 0.4, 1)
    Up, _ = heatbath.gauge_update(U, lat, 5.3, 1, 0, 77, 1, colour_mask=1)
    eta = estimator.global_noise(lat, 0, 5, 3)
    dense = estimator.ln_factor_dense(U, Up, eta[lat.black_sites()], lat, KAPPA)
    delta = estimator.ln_factor_delta(U, Up, eta, lat, KAPPA, tol=1e-14)
    assert abs(dense - delta) < 1e-8
    # no change, no log ratio
    assert abs(estimator.ln_factor_delta(U, U, eta, lat, KAPPA)) < 1e-11


def test_schur_eigenvalues_equal_to_one():
    """Sec. 4: M - 1 = Dhat'^{-1}(Dhat - Dhat') ends in D_wb, so at least
    dim - 2 rank(D_wb) eigenvalues of M^dag M are exactly one."""
    dims = (8, 2, 2, 2)
    lat = geometry.Lattice(dims, (4, 2, 2, 2), active_mode="paper")
    U = synthetic.random_gauge(dims, 0.4, 3)
    rs = np.random.default_rng(4)
    Up = np.array(U)
    kick = synthetic.random_su3((int(lat.active.sum()),), 0.5, rs)
    Up[lat.active] = Up[lat.active] @ kick
    D = dirac.dense_D(U, lat, KAPPA)
    Dp = dirac.dense_D(Up, lat, KAPPA)
    A, B, C, E = dirac.dd_blocks(D, lat)
    M = np.linalg.solve(dirac.dense_schur(Dp, lat), dirac.dense_schur(D, lat))
    ev = np.linalg.eigvalsh(M.conj().T @ M)
    r = np.linalg.matrix_rank(C, tol=1e-10)
    ones = np.sum(np.abs(ev - 1) < 1e-10)
    assert r < M.shape[0] // 2          # the bound is not empty
    assert ones >= M.shape[0] - 2 * r
    assert np.sum(np.abs(ev - 1) > 1e-6) > 0   # and the change is seen


# ---------------------------------------------------------------- interpolation
def test_geodesic_closed_form():
    """U' = U exp(i eps H): the path is U exp(i t eps H) (eigen-phases |.| < pi)."""
    rs = np.random.default_rng(5)
    n = 500
    U = synthetic.random_su3((n,), 1.0, rs)
    lam = synthetic.gell_mann()
    w = rs.standard_normal((n, 8))
    H = np.einsum("nk,kij->nij", w, lam)
    ev, vec = np.linalg.eigh(H)
    eps = 0.9 / np.max(np.abs(ev), axis=1)          # keep all phases inside (-pi, pi)
    def expm(t):
        return np.einsum("nik,nk,njk->nij", vec, np.exp(1j * t * eps[:, None] * ev), np.conj(vec))
    Up = U @ expm(1.0)
    for t in (0.0, 0.25, 1 / 3, 0.5, 0.9, 1.0):
        Ut = interp.interpolate(U[:, None], Up[:, None], t)[:, 0]
        assert np.max(np.abs(Ut - U @ expm(t))) < 1e-12
        assert np.max(np.abs(np.linalg.det(Ut) - 1)) < 1e-12
        assert np.max(np.abs(Ut @ np.conj(np.transpose(Ut, (0, 2, 1))) - np.eye(3))) < 1e-12


def test_geodesic_large_changes_and_reversal():
    rs = np.random.default_rng(6)
    n = 2000
    U = synthetic.random_su3((n, 1), 3.0, rs)
    Up = synthetic.random_su3((n, 1), 3.0, rs)     # far apart, phases near pi occur
    N = 7
    path = [interp.interpolate(U, Up, i / N) for i in range(N + 1)]
    assert np.array_equal(path[0], U) and np.array_equal(path[-1], Up)
    steps = []
    for i in range(N):
        a, b = path[i][:, 0], path[i + 1][:, 0]
        assert np.max(np.abs(np.linalg.det(b) - 1)) < 1e-11
        steps.append(np.linalg.norm(a - b, axis=(1, 2)))
    steps = np.array(steps)
    # geodesic: equal steps along the path
    assert np.max(np.abs(steps - steps[0])) < 1e-10
    # the reversed path visits the same links
    for i in range(1, N):
        back = interp.interpolate(Up, U, (N - i) / N)
        assert np.max(np.abs(back - path[i])) < 1e-10


def test_interpolation_factorisation_telescopes():
    """Eq. param: prod_i det(M_i^dag M_i) = det(M^dag M)."""
    dims = (4, 4, 4, 4)
    lat = geometry.Lattice(dims, (2, 2, 2, 2))
    U = synthetic.random_gauge(dims, 0.4, 1)
    Up, _ = heatbath.gauge_update(U, lat, 5.3, 1, 0, 8, 2, colour_mask=3)
    N = 3
    tot = 0.0
    for i in range(N):
        tot += estimator.exact_ln_ratio_schur(interp.interpolate(U, Up, i / N, lat.active),
                                              interp.interpolate(U, Up, (i + 1) / N, lat.active), lat, KAPPA)
    assert abs(tot - estimator.exact_ln_ratio_schur(U, Up, lat, KAPPA)) < 1e-9


# ------------------------------------------------------------------- acceptance
@pytest.mark.parametrize("sigma2", [0.1, 1.0, 4.0, 16.0])
def test_gaussian_acceptance_law(sigma2):
    """Eq. acceptance: Delta ~ N(sigma^2/2, sigma^2) gives <P_acc> = erfc(sqrt(sigma^2/8))."""
    n = 400000
    d = np.random.default_rng(int(sigma2 * 10)).normal(sigma2 / 2, math.sqrt(sigma2), n)
    u = rng.accept_uniform(np.arange(n, dtype=np.uint64), rng.PURPOSE_GLOBAL_ACCEPT, 31, 7)
    acc = accept.accept_decision(-d, u)
    p = accept.gaussian_acceptance(sigma2)
    assert abs(acc.mean() - p) < 5 * math.sqrt(p * (1 - p) / n)
    assert abs(np.minimum(1, np.exp(-d)).mean() - p) < 5 * math.sqrt(0.25 / n)


# --------------------------------------------------------------------- heatbath
@pytest.mark.parametrize("alpha", [0.7, 4.0, 25.0])
def test_kennedy_pendleton_density(alpha):
    n = 60000
    el = np.arange(n, dtype=np.uint64)
    x0, ok = heatbath.kp_sample_x0(np.full(n, alpha), el, 0, 99, 3)
    assert ok.all()
    dens = lambda x: math.sqrt(max(0.0, 1 - x * x)) * math.exp(alpha * (x - 1))
    Z = integrate.quad(dens, -1, 1, limit=200)[0]
    xs = np.sort(x0)
    grid = np.linspace(-1, 1, 41)
    cdf = np.array([integrate.quad(dens, -1, g, limit=200)[0] / Z for g in grid])
    emp = np.searchsorted(xs, grid, side="right") / n
    assert np.max(np.abs(emp - cdf)) < 1.63 / math.sqrt(n) * 1.5   # KS, 1% level, margin


def test_overrelaxation_keeps_action():
    dims = (4, 4, 4, 4)
    lat = geometry.Lattice(dims, (2, 2, 2, 2))
    U = synthetic.random_gauge(dims, 0.5, 3)
    allmask = np.ones((lat.V, 4), dtype=bool)
    S0 = heatbath.wilson_action(U, lat, 5.3)
    # one OR sweep alone: run with n_hb=0 through the group routine
    V = np.array(U)
    for a in range(4):
        for par in (0, 1):
            sites = np.nonzero(lat.parity == par)[0]
            heatbath.heatbath_group(V, lat, sites, a, 5.3, 0, 1, 1, overrelax=True)
    assert abs(heatbath.wilson_action(V, lat, 5.3) - S0) < 1e-10 * abs(S0)
    assert np.max(np.abs(V - U)) > 1e-3


def test_heatbath_changes_only_active_links_and_stays_su3():
    dims = (8, 8, 8, 8)
    lat = geometry.Lattice(dims, (4, 4, 4, 4))
    U = synthetic.random_gauge(dims, 0.3, 2)
    Up, fails = heatbath.gauge_update(U, lat, 5.3, 1, 1, 5, 9)
    changed = np.any(np.abs(Up - U) > 0, axis=(2, 3))
    assert np.all(changed <= lat.active) and changed.sum() == lat.active.sum()
    assert fails == 0
    a = Up[lat.active]
    assert np.max(np.abs(a @ np.conj(np.transpose(a, (0, 2, 1))) - np.eye(3))) < 1e-12
    assert np.max(np.abs(np.linalg.det(a) - 1)) < 1e-12


@pytest.mark.slow
def test_strong_coupling_plaquette():
    """At small beta, <Re tr U_P / 3> = beta/18 + beta^2/216 + O(beta^3) (SU(3))."""
    dims = (4, 4, 4, 4)
    lat = geometry.Lattice(dims, (2, 2, 2, 2))
    beta = 1.0
    U = synthetic.random_gauge(dims, 3.0, 4)
    allmask = np.ones((lat.V, 4), dtype=bool)
    vals = []
    for sweep in range(60):
        U, _ = heatbath.gauge_update(U, lat, beta, 1, 0, 1234, sweep, active=allmask)
        if sweep >= 10:
            vals.append(heatbath.plaquette_mean(U, lat))
    ref = beta / 18 + beta ** 2 / 216
    err = np.std(vals) / math.sqrt(len(vals)) * 2
    assert abs(np.mean(vals) - ref) < 5 * err + 2e-3


def test_block_filter_delta_form_equals_definition():
    """Per block: -(|D_b'^{-1} D_b eta_b|^2 - |eta_b|^2) with dense D_b, summed
    over the interpolation factors, equals the delta form of the oracle."""
    dims = (4, 4, 4, 4)
    lat = geometry.Lattice(dims, (2, 2, 2, 2))
    U = synthetic.random_gauge(dims, 0.4, 1)
    Up, _ = heatbath.gauge_update(U, lat, 5.3, 1, 0, 77, 1, colour_mask=2)
    n = 2
    got = estimator.block_ln_ratios(U, Up, lat, KAPPA, n, 5, 3, colour_mask=2)
    ref = np.zeros(lat.nblocks)
    for i in range(n):
        Ui = interp.interpolate(U, Up, i / n, lat.active)
        Uj = interp.interpolate(U, Up, (i + 1) / n, lat.active)
        eta = estimator.block_noise(lat, i, 5, 3)
        for blk in lat.white_blocks:
            e = eta[lat.block_sites_of(blk)].reshape(-1)
            Me = np.linalg.solve(dirac.dense_dirichlet_block(Uj, lat, KAPPA, blk),
                                 dirac.dense_dirichlet_block(Ui, lat, KAPPA, blk) @ e)
            ref[blk] += -(np.vdot(Me, Me).real - np.vdot(e, e).real)
    assert np.max(np.abs(got - ref)) < 1e-9
    assert np.all(got[lat.black_blocks] == 0)
