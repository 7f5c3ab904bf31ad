"""GPU parity of the proposal, the block filter, the global stochastic
estimate and the acceptance steps, through the C ABI, against the oracle.

Tolerances:
  * heat-bath links: 1e-12 absolute (same Philox words; libm log/cos may
    differ by an ulp, which a chain of FP64 products amplifies mildly);
  * block log-ratios: 1e-8 absolute (block solves to 1e-12 relative residual);
  * global log-ratios: |d ln| <= max(1e-8, 20 (|eta| + |d|) ||D'^{-1}|| 1e-10 ||s||)
    from the global solve's relative residual 1e-10 (the other errors are
    below it); ||D'^{-1}|| from the dense smallest singular value (4^4);
    on 8^4 and 16^4 the plain FP64 path with solves to 1e-14 is held to
    1e-8 absolute, the mixed path to the bound of its residuals, both
    against oracle values written by tests/golden/make_global_estimates.py;
  * accept flags and restored links: exact wherever |ln u - ln r| > 1e-8.
"""
import numpy as np
import pytest

from oracle import accept, dirac, estimator, geometry, heatbath, rng
from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return lib_api()


@pytest.mark.parametrize("dims,block,mode,cm", [((8, 8, 8, 8), (4, 4, 4, 4), "paper", 3),
                                               ((4, 4, 4, 4), (2, 2, 2, 2), "intra", 1),
                                               ((4, 4, 4, 4), (2, 2, 2, 2), "intra", 2)])
def test_heatbath_matches_oracle(api, dims, block, mode, cm):
    lat = geometry.Lattice(dims, block, active_mode=mode)
    U = synthetic.random_gauge(dims, 0.3, 2)
    code = {"paper": api.DD_ACTIVE_PAPER, "intra": api.DD_ACTIVE_INTRA}[mode]
    h = api.dd_init(dims, block, 0.13, active_mode=code)
    Ud = dev(U)
    api.dd_gauge_update(h, Ud, cm, 5.3, 2, 1, 42, 7)
    ref, fails = heatbath.gauge_update(U, lat, 5.3, 2, 1, 42, 7, colour_mask=cm)
    got = host(Ud)
    assert np.max(np.abs(got - ref)) < 1e-12
    st, hbf = api.dd_status(h)
    assert st == 0 and hbf == fails


def _block_case(api, dims, block, mode, cm, n, eps=0.3, kappa=0.13):
    lat = geometry.Lattice(dims, block, active_mode=mode)
    code = {"paper": api.DD_ACTIVE_PAPER, "intra": api.DD_ACTIVE_INTRA, "inner6": api.DD_ACTIVE_INNER6}[mode]
    h = api.dd_init(dims, block, kappa, active_mode=code, max_rhs=n)
    U = synthetic.random_gauge(dims, eps, 2)
    Up, _ = heatbath.gauge_update(U, lat, 5.3, 1, 0, 11, 3, colour_mask=cm)
    return lat, h, U, Up


@pytest.mark.parametrize("dims,block,mode,cm,n", [((4, 4, 4, 4), (2, 2, 2, 2), "intra", 1, 1),
                                                 ((4, 4, 4, 4), (2, 2, 2, 2), "intra", 2, 3),
                                                 ((8, 8, 8, 8), (4, 4, 4, 4), "paper", 3, 2)])
@pytest.mark.parametrize("masked", [0, 1])
def test_block_filter_stochastic(api, dims, block, mode, cm, n, masked):
    """Both forms of the filter: the persistent per-block launch and the
    batched whole-lattice Dirichlet solves."""
    lat, h, U, Up = _block_case(api, dims, block, mode, cm, n)
    api.dd_set_tuning(h, filter_masked=masked)
    kappa = 0.13
    Upd = dev(Up)
    ln_b, acc = api.dd_block_filter(h, dev(U), Upd, cm, api.DD_FILTER_STOCHASTIC, n, 99, 5)
    ref = estimator.block_ln_ratios(U, Up, lat, kappa, n, 99, 5, colour_mask=cm)
    got = host(ln_b)
    assert np.max(np.abs(got - ref)) < 1e-8, np.max(np.abs(got - ref))
    racc, lu = accept.block_accept(ref, 99, 5, cm, lat.block_colour)
    clear = np.abs(lu - ref) > 1e-8
    gacc = host(acc).astype(bool)
    assert np.array_equal(gacc[clear], racc[clear])
    # rejected blocks restored exactly, accepted blocks keep the proposal
    ref_U = accept.restore_rejected_blocks(Up, U, lat, gacc)
    assert np.array_equal(host(Upd), ref_U)
    assert api.dd_status(h)[0] == 0


def _dinv_norm(U, lat, kappa):
    D = dirac.dense_D(U, lat, kappa)
    return 1.0 / np.linalg.svd(D, compute_uv=False)[-1]


@pytest.mark.parametrize("prec,krylov", [(0, 0), (1, 0), (2, 0), (2, 1), (2, 2)])
@pytest.mark.parametrize("n,mode", [(1, "factors"), (3, "factors"), (2, "replicas")])
def test_global_estimate_small(api, prec, krylov, n, mode):
    dims, block, kappa = (4, 4, 4, 4), (2, 2, 2, 2), 0.12
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.4, 1)
    Up, _ = heatbath.gauge_update(U, lat, 5.3, 1, 0, 77, 1, colour_mask=3)
    h = api.dd_init(dims, block, kappa, max_rhs=n, inner_prec=prec, krylov=krylov)
    m = api.DD_EST_FACTORS if mode == "factors" else api.DD_EST_REPLICAS
    got = host(api.dd_det_ratio_estimate(h, dev(U), dev(Up), n, 5, 3, m))
    ref = estimator.det_ratio_estimate(U, Up, lat, kappa, n, 5, 3, mode=mode, tol=1e-14)
    dn = _dinv_norm(Up, lat, kappa)
    for i in range(n):
        eta = estimator.global_noise(lat, i, 5, 3)
        if mode == "factors":
            from oracle.interp import interpolate
            Ui = interpolate(U, Up, i / n, lat.active)
            Uj = interpolate(U, Up, (i + 1) / n, lat.active)
        else:
            Ui, Uj = U, Up
        s = estimator.delta_source(Ui, Uj, eta, lat, kappa)
        d = np.linalg.norm(s) * dn
        bound = max(1e-8, 20 * (np.linalg.norm(eta) + d) * dn * 1e-10 * np.linalg.norm(s))
        assert abs(got[i] - ref[i]) <= bound, (i, got[i], ref[i], bound)
    assert api.dd_status(h)[0] == 0


def golden_case(name):
    """Oracle values of the global estimate written by
    tests/golden/make_global_estimates.py (solves to 1e-14, oracle only)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "global_estimates.json")
    with open(path) as f:
        return json.load(f)[name]


def golden_fields(w):
    """The same seeded fields as the golden script: U' = R U on the active links."""
    lat = geometry.Lattice(tuple(w["dims"]), tuple(w["block"]))
    U = synthetic.random_gauge(tuple(w["dims"]), w["eps"], w["seed"])
    R = synthetic.random_gauge(tuple(w["dims"]), w["kick_eps"], w["kick_seed"])
    Up = np.array(U, copy=True)
    Up[lat.active] = R[lat.active] @ U[lat.active]
    return lat, U, Up


def worst_case_bound(f, tol_global, tol_block):
    """|d ln r_i| from the solves' relative residuals (Cauchy-Schwarz, factor
    10 for the operator norms of the Schur pieces and a safety factor 10):
      global solve:  2 (|eta| + |delta|) ||D'^{-1}|| tol_global ||s||
      block solves:  2 (|eta| + |delta|) ||D'^{-1}|| 10 tol_block |eta|
    with |delta| <= ||D'^{-1}|| ||s||."""
    dn, s, e = f["dinv_norm"], f["s_norm"], f["eta_norm"]
    pre = 2.0 * (e + dn * s) * dn
    g, b = pre * tol_global * s, pre * 10.0 * tol_block * e
    return 10.0 * (g + b), ("global solve" if g >= b else "block solves")


@pytest.mark.parametrize("name", ["8x4", "16x8"])
def test_global_estimate_fp64_within_1e8(api, name):
    """8^4 (4^4 blocks) and 16^4 (8^4 blocks, 6^4 active sub-blocks): the
    plain FP64 path with every solve to 1e-14 matches the oracle's ln r_i
    (solves to 1e-14) within the 1e-8 absolute tolerance of the log-ratios."""
    gc = golden_case(name)
    w = gc["workload"]
    lat, U, Up = golden_fields(w)
    n = w["n"]
    h = api.dd_init(tuple(w["dims"]), tuple(w["block"]), w["kappa"], max_rhs=n, inner_prec=api.DD_PREC_F64,
                    block_prec=api.DD_PREC_F64, krylov=api.DD_KRYLOV_CGNR, tol_global=1e-14, tol_block=1e-14,
                    maxit=100000)
    got = host(api.dd_det_ratio_estimate(h, dev(U), dev(Up), n, w["noise_seed"], w["ctr"], api.DD_EST_FACTORS))
    for i, f in enumerate(gc["factors"]):
        bound, binds = worst_case_bound(f, 1e-14, 1e-14)
        print(f"{name} factor {i}: ln {got[i]:.12f} oracle {f['ln']:.12f} diff {abs(got[i] - f['ln']):.2e} "
              f"(worst-case bound {bound:.1e}, {binds} term)")
        assert abs(got[i] - f["ln"]) <= 1e-8, (i, got[i], f["ln"])
    assert api.dd_status(h)[0] == 0


@pytest.mark.parametrize("name,krylov", [("8x4", 0), ("8x4", 1), ("16x8", 1)])
def test_global_estimate_mixed_within_bound(api, name, krylov):
    """The mixed path (FP16 storage, FP32 inner solver, FP64 defect
    correction; global residual 1e-10, block residual 1e-12) against the
    oracle, within the bound that those residuals allow (computed from the
    oracle's |eta|, ||s|| and ||D'^{-1}||; the test prints which term binds)."""
    gc = golden_case(name)
    w = gc["workload"]
    lat, U, Up = golden_fields(w)
    n = w["n"]
    h = api.dd_init(tuple(w["dims"]), tuple(w["block"]), w["kappa"], max_rhs=n, inner_prec=api.DD_PREC_F16,
                    krylov=krylov, tol_global=1e-10, tol_block=1e-12)
    got = host(api.dd_det_ratio_estimate(h, dev(U), dev(Up), n, w["noise_seed"], w["ctr"], api.DD_EST_FACTORS))
    for i, f in enumerate(gc["factors"]):
        bound, binds = worst_case_bound(f, 1e-10, 1e-12)
        bound = max(1e-8, bound)
        print(f"{name} krylov {krylov} factor {i}: diff {abs(got[i] - f['ln']):.2e} bound {bound:.1e} ({binds})")
        assert abs(got[i] - f["ln"]) <= bound, (i, got[i], f["ln"], bound)
    assert api.dd_status(h)[0] == 0


def test_global_accept(api):
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    h = api.dd_init(dims, block, 0.12)
    U0 = synthetic.random_gauge(dims, 0.4, 1)
    U1 = synthetic.random_gauge(dims, 0.4, 2)
    import torch
    for ctr in range(6):
        ln = torch.tensor([-0.3 * ctr, 0.1], dtype=torch.float64, device="cuda")
        Ud = dev(U1)
        acc, margin = api.dd_global_accept(h, Ud, dev(U0), ln, 17, ctr)
        ref_acc, lu = accept.global_accept(float(ln.sum()), 17, ctr)
        assert bool(host(acc)[0]) == ref_acc
        assert abs(float(host(margin)[0]) - (float(ln.sum()) - lu)) < 1e-15
        assert np.array_equal(host(Ud), U1 if ref_acc else U0)
