"""Support for the pins of the oracle's Markov-chain composition.

The chain functions of the oracle (``oracle.chain.hierarchical_step``,
``oracle.recursive.recursive_step``) compose a proposal, block filters with
their accept/restore steps and the global estimate.  To pin the composition
against the paper, the tests replace the random parts that are pinned
elsewhere by fixed stand-ins:

* ``FixedProposal``: the proposal changes exactly the active links of the
  selected block colours to those of a given field (a heat-bath sweep changes
  the same links, Sec. 3: only active links are updated);
* ``ForcedDecisions``: block accept/reject decisions given by the test;
* ``Recorder``: records the arguments of the estimator calls and returns
  fixed values (the estimators themselves are pinned by their own tests).

The ``*_sample`` functions run one chain step for one random-stream seed and
are executed in worker processes (start method ``spawn``) by the Monte Carlo
pins; they patch the oracle modules of the worker only.
"""
import numpy as np

from oracle import accept, chain, estimator, heatbath, recursive
from paper_1112_1243_gb300 import synthetic


def kicked(U, lat, mask, eps, seed):
    """U' = R U on the links of `mask`, R = exp(i eps H) with random H."""
    R = synthetic.random_gauge(lat.dims, eps, seed)
    Up = np.array(U, copy=True)
    Up[mask] = R[mask] @ U[mask]
    return Up


def colour_sel(lat, colour_mask):
    """Sites of the blocks whose colour is in colour_mask."""
    return np.isin(lat.colour, [c for c in (0, 1) if colour_mask >> c & 1])


class FixedProposal:
    """Stand-in for heatbath.gauge_update: the active links of the selected
    block colours take the values of `target`; everything else is kept."""

    def __init__(self, target):
        self.target = target
        self.calls = []

    def __call__(self, U, lat, beta, n_hb, n_or, seed, ctr, colour_mask=3, active=None):
        act = lat.active if active is None else active
        self.calls.append((np.array(U, copy=True), colour_mask, ctr))
        out = np.array(U, copy=True)
        m = act & colour_sel(lat, colour_mask)[:, None]
        out[m] = self.target[m]
        return out, 0


class ForcedDecisions:
    """Stand-in for a block accept step: `pattern[k]` (one bool per block) is
    the decision of the k-th call for the blocks of the selected colours;
    blocks of other colours are reported accepted (their links are not
    touched), as in the oracle."""

    def __init__(self, patterns):
        self.patterns = list(patterns)
        self.k = 0

    def __call__(self, ln_rb, seed, ctr, colour_mask=3, block_colour=None):
        pat = np.asarray(self.patterns[min(self.k, len(self.patterns) - 1)], dtype=bool)
        self.k += 1
        acc = pat.copy()
        if block_colour is not None:
            sel = np.isin(block_colour, [c for c in (0, 1) if colour_mask >> c & 1])
            acc = np.where(sel, acc, True)
        return acc, np.zeros(len(pat))


class Recorder:
    """Stand-in for an estimator: records (U, Up) and the keyword/positional
    arguments, returns `value(n)`."""

    def __init__(self, value):
        self.value = value
        self.calls = []

    def __call__(self, U, Up, lat, kappa, n, seed, ctr, **kw):
        self.calls.append(dict(U=np.array(U, copy=True), Up=np.array(Up, copy=True), n=n, seed=seed, ctr=ctr, kw=kw))
        return self.value(n)


def restore_by_definition(U_new, U_old, lat, accepted):
    """Sec. 3 / Eq. 4step: the links of a rejected block go back to their old
    values; only active links can differ.  Written link by link."""
    out = np.array(U_new, copy=True)
    for s in range(lat.V):
        if accepted[lat.block_id[s]]:
            continue
        for a in range(4):
            if lat.active[s, a]:
                out[s, a] = U_old[s, a]
    return out


# ------------------------------------------------------------ Monte Carlo
def _threads_one():
    import os
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def global_sample(args):
    """One hierarchical step with the fixed proposal `target` and every block
    accepted; returns the per-factor global log-ratios of the record."""
    U0, lat, target, kappa, n_global, seed, tol = args
    heatbath.gauge_update = FixedProposal(target)
    accept.block_accept = ForcedDecisions([np.ones(lat.nblocks, dtype=bool)])
    _, rec = chain.hierarchical_step(U0, lat, kappa, 5.3, 1, 1, n_global, seed, 0, filter_mode="exact", tol=tol)
    return np.asarray(rec["ln_global"])


def block_schur_sample(args):
    """One recursive step with the fixed proposal `target`, no sub-block
    factor (every sub-block then accepts: ln u < 0) and no global factor;
    returns the per-block step-2 log-ratios of the record."""
    U0, tl, target, kappa, n_block, seed, tol = args
    heatbath.gauge_update = FixedProposal(target)
    _, rec = recursive.recursive_step(U0, tl, kappa, 5.3, 1, 0, n_block, 0, seed, 0, tol=tol)
    return np.asarray(rec["block"][0][0])


def run_pool(fn, argv, workers=None):
    """Map fn over argv in `spawn` worker processes (one BLAS thread each)."""
    import multiprocessing as mp
    import os
    n = workers or max(1, min(8, os.cpu_count() or 1))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    _threads_one()
    try:
        with mp.get_context("spawn").Pool(n) as pool:
            return pool.map(fn, argv, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
