"""Metropolis acceptance steps (oracle).

Paper Sec. 2: a proposal followed by acceptance with probability
min{1, P_i(s')/P_i(s)} = min{1, exp(-Delta_i)}; several such steps in a row
form the hierarchy (Eq. factor and the steps after it).  Realised as
"accept iff ln u < ln r" with u uniform in (0, 1): P(accept) = min(1, r).

Eq. acceptance: for Gaussian Delta with variance sigma^2 the mean acceptance
is erfc(sqrt(sigma^2 / 8)).  The mean of Delta is not stated; the law holds
for mean sigma^2/2, which is what <exp(-Delta)> = 1 (the estimator being
unbiased for a ratio of normalised distributions) implies.
"""
import math

import numpy as np

from . import rng


def accept_decision(ln_r, u):
    """True where ln u < ln r (strict)."""
    return np.log(u) < ln_r


def block_accept(ln_rb, seed, ctr, colour_mask=3, block_colour=None):
    """Per-block decisions; blocks of unselected colours are not touched
    (reported as accepted: their links did not change)."""
    nb = len(ln_rb)
    u = rng.accept_uniform(np.arange(nb, dtype=np.uint64), rng.PURPOSE_BLOCK_ACCEPT, seed, ctr)
    acc = accept_decision(np.asarray(ln_rb), u)
    if block_colour is not None:
        sel = np.isin(block_colour, [c for c in (0, 1) if colour_mask >> c & 1])
        acc = np.where(sel, acc, True)
    return acc, np.log(u)


def global_accept(ln_r_total, seed, ctr):
    u = rng.accept_uniform(np.zeros(1, dtype=np.uint64), rng.PURPOSE_GLOBAL_ACCEPT, seed, ctr)[0]
    return bool(math.log(u) < ln_r_total), math.log(u)


def restore_rejected_blocks(U_new, U_old, lat, accepted):
    """Put back U_old on the active links of rejected blocks."""
    out = np.array(U_new, copy=True)
    rej = ~np.asarray(accepted)[lat.block_id]
    m = lat.active & rej[:, None]
    out[m] = U_old[m]
    return out


def gaussian_acceptance(sigma2):
    """erfc(sqrt(sigma^2 / 8)), Eq. acceptance."""
    return math.erfc(math.sqrt(sigma2 / 8.0))
