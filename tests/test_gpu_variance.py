"""Thermalisation with the heat-bath on every link (active set "all")
against the oracle, and a small variance scan of the global step (Sec. 5,
"Exact acceptance rate") end to end on the GPU."""
import numpy as np
import pytest

from oracle import geometry, heatbath
from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return lib_api()


def test_heatbath_all_links_matches_oracle(api):
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    lat = geometry.Lattice(dims, block, active_mode="all")
    U = synthetic.random_gauge(dims, 0.5, 9)
    h = api.dd_init(dims, block, 0.12, active_mode=api.DD_ACTIVE_ALL)
    assert api.dd_get_maps(h)["active"].all()
    Ud = dev(U)
    api.dd_gauge_update(h, Ud, 3, 5.8, 1, 1, 3, 4)
    ref, fails = heatbath.gauge_update(U, lat, 5.8, 1, 1, 3, 4, colour_mask=3)
    assert np.max(np.abs(host(Ud) - ref)) < 1e-12


def test_variance_scan_small(api):
    import torch
    from paper_1112_1243_gb300 import variance
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    U = torch.from_numpy(synthetic.unit_gauge(dims)).to("cuda")
    plaq = variance.thermalise(api, dims, block, 5.8, 20, 1, 5, U)
    assert 0.3 < plaq < 1.0
    h = api.dd_init(dims, block, 0.13, max_rhs=2, inner_prec=api.DD_PREC_F16, krylov=api.DD_KRYLOV_BICGSTAB)
    res = variance.variance_scan(api, h, U, 5.8, [1, 2], 4, 7, n_block=2)
    assert len(res["rows"]) == 2
    for r in res["rows"]:
        assert np.isfinite(r["var"]) and r["var"] >= 0
    assert 0.0 <= res["acceptance_exact"] <= 1.0
    assert api.dd_status(h)[0] == 0
