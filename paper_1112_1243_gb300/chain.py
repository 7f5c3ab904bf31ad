"""The hierarchical Markov step (Sec. 5, the three-step algorithm; Eq. 4step
steps 0, 1 and 3) on top of the C ABI.

The step itself runs in libdd.so (dd_chain_step): U0 <- U; n_inner times
proposal on the active links + block filter; stochastic global step and
accept.  Counters of the random streams follow the oracle's convention:
ctr = step << 20 | iteration << 4 | colour pass for the proposal and the
block filter of an iteration, ctr = step << 20 | n_inner << 4 for the global
step.  A step can be recorded once as a CUDA graph (capture) and replayed
as step k with the counters advanced by k << 20 (step_graph).
"""
import torch

from . import api


def counter(step, iteration, colour_pass):
    return (int(step) << 20) | (int(iteration) << 4) | int(colour_pass)


class HierarchicalStep:
    """State and buffers of one Markov chain on one handle.

    n_inner proposal/filter iterations per global step; n_block interpolation
    factors in the block filter, n_global in the global step; colour passes
    1 and 2 (black, white) when the active set is "intra", one pass otherwise.
    On a handle with sub-blocks, n_schur > 0 adds the blocks' Schur filter
    (Eq. 4step step 2) after the sub-block filter of every iteration.
    gauge_fix_sweeps > 0 fixes the proposal relative to the old field before
    the global estimate (Sec. 4).
    """

    def __init__(self, h, beta, n_inner=1, n_block=4, n_global=12, n_or=0, seed=1,
                 filter_mode=api.DD_FILTER_STOCHASTIC, intra=False, n_schur=0, gauge_fix_sweeps=0):
        self.h = h
        self.beta = float(beta)
        self.n_inner = int(n_inner)
        self.n_block = int(n_block)
        self.n_global = int(n_global)
        self.n_or = int(n_or)
        self.seed = int(seed)
        self.filter_mode = int(filter_mode)
        self.passes = [1, 2] if intra else [3]
        dev = h.workspace.device
        shape = (h.V, 4, 3, 3)
        self.U0 = torch.empty(shape, dtype=torch.complex128, device=dev)
        self.Up = torch.empty(shape, dtype=torch.complex128, device=dev)
        # step 1 per smallest block; step 2 (handles with sub-blocks) per block
        self.ln_b = torch.zeros(h.nfine, dtype=torch.float64, device=dev)
        self.acc_b = torch.zeros(h.nfine, dtype=torch.uint8, device=dev)
        self.n_schur = int(n_schur)
        self.ln_bs = torch.zeros(h.nblocks, dtype=torch.float64, device=dev)
        self.acc_bs = torch.zeros(h.nblocks, dtype=torch.uint8, device=dev)
        self.ln_g = torch.zeros(self.n_global, dtype=torch.float64, device=dev)
        self.acc_g = torch.zeros(1, dtype=torch.uint8, device=dev)
        self.margin = torch.zeros(1, dtype=torch.float64, device=dev)
        self.params = api.dd_chain_params()
        self.params.beta = self.beta
        self.params.n_inner = self.n_inner
        self.params.n_block = self.n_block
        self.params.n_global = self.n_global
        self.params.n_hb = 1
        self.params.n_or = self.n_or
        self.params.filter_mode = self.filter_mode
        self.params.colour_passes = len(self.passes)
        self.params.n_schur = self.n_schur
        self.params.gauge_fix_sweeps = int(gauge_fix_sweeps)
        self.params.seed = self.seed
        self.buffers = {"U0": self.U0, "Up": self.Up, "ln_b": self.ln_b, "acc_b": self.acc_b, "ln_g": self.ln_g,
                        "acc_g": self.acc_g, "margin": self.margin, "ln_bs": self.ln_bs, "acc_bs": self.acc_bs}
        self.graph = None
        self.graph_U = None

    def step(self, U, k):
        """Advance the chain state U (device tensor, updated in place) by one
        global step with step index k."""
        api.dd_chain_step(self.h, U, self.params, self.buffers, k)
        return self.ln_g, self.acc_g

    def capture(self, U):
        """Record one step on U (step index 0) as a CUDA graph; nothing runs."""
        api.dd_graph_begin(self.h)
        try:
            api.dd_chain_step(self.h, U, self.params, self.buffers, 0)
        finally:
            g = api.dd_graph_end(self.h)
        self.graph, self.graph_U = g, U
        return g

    def step_graph(self, k):
        """Replay the recorded step as step k on the tensor given to capture."""
        api.dd_graph_launch(self.graph, int(k) << 20)
        return self.ln_g, self.acc_g

    def step_host(self, U_host, U_dev, k, ln_host, acc_host):
        """End-to-end form: U_host (pinned) -> device, one step, the per-factor
        log-ratios, the decision and the new configuration back to the host."""
        U_dev.copy_(U_host, non_blocking=True)
        ln, acc = self.step(U_dev, k)
        ln_host.copy_(ln, non_blocking=True)
        acc_host.copy_(acc, non_blocking=True)
        U_host.copy_(U_dev, non_blocking=True)
        return ln_host, acc_host
