"""Host driver of the hierarchical Markov step (Sec. 5, "3-step algorithm";
Eq. 4step steps 0, 1 and 3), on top of the C ABI.

Only control flow lives here: every step of the computation is a call into
libdd.so.  Counters of the random streams follow the oracle's convention:
ctr = step << 20 | iteration << 4 | colour pass for the proposal and the
block filter of an iteration, ctr = step << 20 | n_inner << 4 for the global
step.
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
    """

    def __init__(self, h, beta, n_inner=1, n_block=4, n_global=12, n_or=0, seed=1,
                 filter_mode=api.DD_FILTER_STOCHASTIC, intra=False):
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
        self.ln_b = torch.zeros(h.nblocks, dtype=torch.float64, device=dev)
        self.acc_b = torch.zeros(h.nblocks, dtype=torch.uint8, device=dev)
        self.ln_g = torch.zeros(self.n_global, dtype=torch.float64, device=dev)
        self.acc_g = torch.zeros(1, dtype=torch.uint8, device=dev)
        self.margin = torch.zeros(1, dtype=torch.float64, device=dev)

    def step(self, U, k):
        """Advance the chain state U (device tensor, updated in place) by one
        global step with step index k."""
        h = self.h
        self.U0.copy_(U)
        for it in range(self.n_inner):
            for p, cm in enumerate(self.passes):
                ctr = counter(k, it, p)
                self.Up.copy_(U)
                api.dd_gauge_update(h, self.Up, cm, self.beta, 1, self.n_or, self.seed, ctr)
                api.dd_block_filter(h, U, self.Up, cm, self.filter_mode, self.n_block, self.seed, ctr,
                                    self.ln_b, self.acc_b)
                U.copy_(self.Up)
        ctr = counter(k, self.n_inner, 0)
        api.dd_det_ratio_estimate(h, self.U0, U, self.n_global, self.seed, ctr, api.DD_EST_FACTORS, self.ln_g)
        api.dd_global_accept(h, U, self.U0, self.ln_g, self.seed, ctr, self.acc_g, self.margin)
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
