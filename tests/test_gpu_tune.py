"""Autotuner of the launch shapes: every candidate shape computes the same
operator (the stencil's per-site arithmetic does not depend on the tiling,
so Dslash is bit-identical across shapes), the tuner picks a shape from its
candidate set, and solves and block filters stay correct with it."""
import numpy as np
import pytest

from oracle import dirac, geometry
from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return lib_api()


HOP_SHAPES = [(128, 1), (64, 1), (128, 2), (64, 2)]


def test_dslash_identical_across_shapes(api):
    dims, block, kappa = (8, 8, 8, 12), (4, 4, 4, 6), 0.13
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.3, 4)
    psi = synthetic.random_spinor(dims, 8, nrhs=3)
    h = api.dd_init(dims, block, kappa, max_rhs=3)
    Ud, pd = dev(U), dev(psi)
    ref = np.stack([dirac.apply_D(U, p, lat, kappa) for p in psi])
    first = {}
    for tpb, spt in HOP_SHAPES:
        for tpb64 in (128, 64):
            api.dd_set_tuning(h, tpb, spt, tpb64, 1, 256, 2)
            for prec in (api.DD_PREC_F64, api.DD_PREC_F16):
                out = dev(np.zeros_like(psi))
                api.dd_apply_D(h, out, pd, Ud, api.DD_OP_D, prec, 3)
                got = host(out)
                assert rel_err(got, ref) < (1e-12 if prec == api.DD_PREC_F64 else 2e-3)
                if prec in first:
                    assert np.array_equal(got, first[prec]), (tpb, spt, tpb64, prec)
                else:
                    first[prec] = got


def test_autotune_picks_candidate_and_stays_correct(api):
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.13
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.3, 2)
    h = api.dd_init(dims, block, kappa, max_rhs=3, krylov=api.DD_KRYLOV_BICGSTAB)
    Ud = dev(U)
    Up = Ud.clone()
    api.dd_gauge_update(h, Up, 3, 5.3, 1, 0, 7, 0)
    rep = api.dd_autotune(h, api.DD_TUNE_HOP | api.DD_TUNE_BLOCK | api.DD_TUNE_NO_CACHE, Ud, Up, reps=4)
    assert (rep["hop_tpb"], rep["hop_spt"]) in HOP_SHAPES
    assert rep["hop64_tpb"] in (64, 128) and rep["hop64_spt"] == 1
    assert (rep["block_tpb"], rep["block_ctas_per_sm"]) in [(256, 2), (256, 1), (128, 2), (128, 4), (64, 4)]
    assert 0 < rep["hop_ms"] <= rep["hop_default_ms"]
    assert 0 < rep["block_ms"] <= rep["block_default_ms"]
    assert rep["filter_masked_ms"] > 0 and rep["filter_masked"] == int(rep["filter_masked_ms"] < rep["block_ms"])
    assert not rep["from_cache"]
    # mixed solve with the tuned shapes
    b = synthetic.random_spinor(dims, 12, nrhs=2)
    x = dev(np.zeros_like(b))
    api.dd_solve(h, x, dev(b), Ud, 2, api.DD_PREC_F16)
    xh = host(x)
    for r in range(2):
        true = np.linalg.norm(b[r] - dirac.apply_D(U, xh[r], lat, kappa)) / np.linalg.norm(b[r])
        assert true <= 1e-10 * 1.01
    # block filter: per-block log-ratios agree across block-solver shapes
    ln_ref = None
    for tpb, ctas, masked in [(256, 2, 0), (128, 4, 0), (64, 4, 0), (256, 2, 1)]:
        api.dd_set_tuning(h, rep["hop_tpb"], rep["hop_spt"], rep["hop64_tpb"], 1, tpb, ctas, masked)
        Un = Up.clone()
        ln_b, acc = api.dd_block_filter(h, Ud, Un, 3, api.DD_FILTER_STOCHASTIC, 2, 11, 3)
        got = host(ln_b)
        if ln_ref is None:
            ln_ref = got
        else:
            # the whole-lattice form meets tol_block relative to all blocks together
            tol = 1e-7 if masked else 1e-9
            assert np.max(np.abs(got - ln_ref)) <= tol * max(1.0, np.max(np.abs(ln_ref))), (tpb, ctas, masked)
    assert api.dd_status(h)[0] == 0
    # the process cache answers a second request without timing
    rep2 = api.dd_autotune(h, api.DD_TUNE_HOP | api.DD_TUNE_BLOCK, Ud, Up, reps=4)
    rep3 = api.dd_autotune(h, api.DD_TUNE_HOP | api.DD_TUNE_BLOCK, Ud, Up, reps=4)
    assert rep3["from_cache"] and (rep3["hop_tpb"], rep3["hop_spt"]) == (rep2["hop_tpb"], rep2["hop_spt"])


def test_instrumentation_counts_and_peaks():
    """dd_alu_peaks gives plausible pipe rates (FP32 FMA far above FP64 FMA);
    dd_solver_stats counts one batched whole-lattice solve of nrhs systems with
    its inner iterations and defect cycles; the kernel timer sees the hop
    kinds of that solve."""
    import torch
    api = lib_api()
    pk = api.dd_alu_peaks()
    assert 0.1 < pk["fp64_fma"] < 20 and 10 < pk["fp32_fma"] < 500 and pk["fp32_fma"] > 10 * pk["fp64_fma"]
    assert 0.05 < pk["fp64_mma"] < 100
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    U = dev(synthetic.random_gauge(dims, 0.3, 5))
    b = dev(synthetic.random_spinor(dims, 6, nrhs=2))
    h = api.dd_init(dims, block, 0.13, max_rhs=2, inner_prec=api.DD_PREC_F16, krylov=api.DD_KRYLOV_BICGSTAB)
    x = torch.zeros_like(b)
    api.dd_kernel_timer(h, 1, 0, 1)
    it, res, _ = api.dd_solve(h, x, b, U, 2, api.DD_PREC_F16)
    st = api.dd_solver_stats(h, 0)
    assert st["solves"] == 1 and st["systems"] == 2 and st["inner_iterations"] == it > 0
    assert st["outer_cycles"] >= 1 and st["site_iterations"] == it * (h.V // 2)
    assert api.dd_solver_stats(h, 1)["solves"] == 0
    ms, cnt, sites = api.dd_kernel_timer(h, 2, 1)
    assert cnt > 0 and ms > 0 and sites > 0
    ms2, cnt2, _ = api.dd_kernel_timer(h, 2, 2)
    assert cnt2 >= 2                                   # FP64 residual hops of the defect correction
    api.dd_kernel_timer(h, 1, 0, 1)                    # reset
    assert api.dd_solver_stats(h, 0)["solves"] == 0
