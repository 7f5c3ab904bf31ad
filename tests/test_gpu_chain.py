"""Accept/reject sequences of the hierarchical step (Sec. 5, 3-step
algorithm) on the GPU against the oracle's chain, with the same random
streams: block and global decisions must be identical wherever
|ln u - ln r| > 1e-8 (closer cases are reported and not compared), and the
configurations must then agree to rounding.
"""
import numpy as np
import pytest

from oracle import chain, geometry
from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return lib_api()


@pytest.mark.parametrize("dims,block,kappa,eps,n_block,n_global,mode,steps", [
    ((4, 4, 4, 4), (2, 2, 2, 2), 0.12, 0.4, 1, 1, "exact", 3),
    ((8, 8, 8, 8), (4, 4, 4, 4), 0.13, 0.3, 2, 2, "stochastic", 2),
])
def test_chain_sequences(api, dims, block, kappa, eps, n_block, n_global, mode, steps):
    from paper_1112_1243_gb300.chain import HierarchicalStep
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, eps, 1)
    h = api.dd_init(dims, block, kappa, max_rhs=max(n_block, n_global), inner_prec=api.DD_PREC_F16)
    fm = api.DD_FILTER_EXACT if mode == "exact" else api.DD_FILTER_STOCHASTIC
    st = HierarchicalStep(h, 5.3, n_inner=1, n_block=n_block, n_global=n_global, seed=1234, filter_mode=fm,
                          intra=lat.active_mode == "intra")
    Ud = dev(U)
    Uo = U.copy()
    near = 0
    for k in range(steps):
        ln_g, acc = st.step(Ud, k)
        Uo, rec = chain.hierarchical_step(Uo, lat, kappa, 5.3, 1, n_block, n_global, 1234, k, filter_mode=mode)
        g_ln = host(ln_g)
        assert np.max(np.abs(g_ln - rec["ln_global"])) < 1e-6
        margin = abs(float(np.sum(rec["ln_global"])) - rec["ln_u"])
        if margin > 1e-8:
            assert bool(host(acc)[0]) == rec["accept"]
        else:
            near += 1
        if near == 0:
            assert np.max(np.abs(host(Ud) - Uo)) < 1e-10
    assert near == 0, f"{near} near-tie decisions (logged, not compared)"
