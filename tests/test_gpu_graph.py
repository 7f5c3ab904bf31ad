"""CUDA-graph capture of the hierarchical step and of a solve: the solver
loops become conditional WHILE nodes evaluated on the device, and a replay
with counter offset k << 20 must reproduce the eager step k bit for bit
(same kernels, same order, same random streams)."""
import numpy as np
import pytest

from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return lib_api()


@pytest.mark.parametrize("dims,block,kappa,eps,krylov,mode", [
    ((8, 8, 8, 8), (4, 4, 4, 4), 0.13, 0.3, 1, "stochastic"),
    ((8, 8, 8, 8), (4, 4, 4, 4), 0.13, 0.3, 0, "stochastic"),
    ((4, 4, 4, 4), (2, 2, 2, 2), 0.12, 0.4, 1, "exact"),
])
def test_graph_replay_matches_eager_steps(api, dims, block, kappa, eps, krylov, mode):
    import torch
    from paper_1112_1243_gb300.chain import HierarchicalStep
    U = synthetic.random_gauge(dims, eps, 3)
    fm = api.DD_FILTER_EXACT if mode == "exact" else api.DD_FILTER_STOCHASTIC
    intra = min(block) <= 2
    steps = 3

    def chain_for():
        h = api.dd_init(dims, block, kappa, max_rhs=4, inner_prec=api.DD_PREC_F16, krylov=krylov)
        return h, HierarchicalStep(h, 5.3, n_inner=1, n_block=2, n_global=3, seed=99, filter_mode=fm, intra=intra)

    ha, ca = chain_for()
    Ua = dev(U)
    eager = []
    for k in range(steps):
        ln, acc = ca.step(Ua, k)
        eager.append((host(ln).copy(), host(acc).copy(), host(ca.ln_b).copy(), host(Ua).copy()))
    assert api.dd_status(ha)[0] == 0

    hb, cb = chain_for()
    Ub = dev(U)
    g = cb.capture(Ub)
    assert api.dd_graph_nodes(g) > 5
    torch.cuda.synchronize()
    # nothing ran during the capture
    assert np.array_equal(host(Ub), U)
    for k in range(steps):
        ln, acc = cb.step_graph(k)
        got = (host(ln), host(acc), host(cb.ln_b), host(Ub))
        for a, b in zip(got, eager[k]):
            assert np.array_equal(a, b), f"step {k}"
    assert api.dd_status(hb)[0] == 0
    api.dd_graph_destroy(g)


def test_graph_of_solve_matches_eager(api):
    """dd_solve recorded once and replayed: same solution bits as the eager
    call, and the residual still meets the target."""
    import torch
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    U = synthetic.random_gauge(dims, 0.3, 5)
    b = synthetic.random_spinor(dims, 6, nrhs=2)
    h = api.dd_init(dims, block, 0.13, max_rhs=2, inner_prec=api.DD_PREC_F16, krylov=1)
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
    # replay again into the same buffers: deterministic
    x_graph.zero_()
    api.dd_graph_launch(g, 0)
    assert np.array_equal(host(x_graph), host(x_eager))
