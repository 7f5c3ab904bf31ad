"""The hierarchical Markov step (oracle).

Paper Sec. 5 (the three-step algorithm): update the active links of a block
decomposition, accept the change block-wise with the block determinant
ratios, repeat this pair "some iterations", then pass the result to the
global acceptance step with the Schur complement (Eq. 4step steps 0, 1, 3;
Sec. 2 for the hierarchy of acceptance steps).

Readings: the number of proposal/filter iterations before the global step
(n_inner) is a parameter; in "intra" mode (2^4 blocks) the proposal and the
block filter run colour by colour (black blocks, then white blocks), since
intra-block links of neighbouring blocks share plaquettes.
Counters of the random streams: ctr = step << 20 | iteration << 4 | pass for
the proposal and filter of iteration `iteration`, colour pass `pass`;
ctr = step << 20 | n_inner << 4 for the global step.
"""
import numpy as np

from . import accept, estimator, gaugefix, heatbath


def counter(step, iteration, colour_pass):
    return (int(step) << 20) | (int(iteration) << 4) | int(colour_pass)


def colour_passes(lat):
    return [1, 2] if lat.active_mode == "intra" else [3]


def hierarchical_step(U, lat, kappa, beta, n_inner, n_block, n_global, seed, step, filter_mode="stochastic",
                      n_or=0, tol=1e-14, gauge_fix_sweeps=0):
    """One global step.  Returns (U_next, record) with the block decisions, the
    per-factor global log-ratios and the global decision."""
    U0 = np.array(U, copy=True)
    Ucur = np.array(U, copy=True)
    rec = {"block": [], "ln_global": None, "accept": None, "ln_u": None}
    for it in range(n_inner):
        for p, cm in enumerate(colour_passes(lat)):
            ctr = counter(step, it, p)
            Up, _ = heatbath.gauge_update(Ucur, lat, beta, 1, n_or, seed, ctr, colour_mask=cm)
            if filter_mode == "exact":
                ln_b = estimator.block_ln_ratios_exact(Ucur, Up, lat, kappa, colour_mask=cm)
            else:
                ln_b = estimator.block_ln_ratios(Ucur, Up, lat, kappa, n_block, seed, ctr, colour_mask=cm, tol=tol)
            acc, lu = accept.block_accept(ln_b, seed, ctr, cm, lat.block_colour)
            rec["block"].append((ln_b, acc, lu))
            Ucur = accept.restore_rejected_blocks(Up, Ucur, lat, acc)
    ctr = counter(step, n_inner, 0)
    if gauge_fix_sweeps > 0:
        # the ratio of the proposal fixed relative to U0 (gauge invariant);
        # the interpolation then runs over every link that differs
        _, Ug, _ = gaugefix.relative_gauge_fix(U0, Ucur, lat, gauge_fix_sweeps)
        ln = estimator.det_ratio_estimate(U0, Ug, lat, kappa, n_global, seed, ctr, tol=tol,
                                          interp_mask=gaugefix.differing_links(U0, Ug))
    else:
        ln = estimator.det_ratio_estimate(U0, Ucur, lat, kappa, n_global, seed, ctr, tol=tol)
    ok, lu = accept.global_accept(float(np.sum(ln)), seed, ctr)
    rec.update(ln_global=ln, accept=ok, ln_u=lu)
    return (Ucur if ok else U0), rec
