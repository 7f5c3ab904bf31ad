"""One level of recursive domain decomposition (oracle).

Paper Eq. ddrec: every block b of the decomposition C is split again into
sub-blocks b' (a checkerboard of black and white sub-blocks inside b), and
    det(D_b) = prod_{b' in C_b} det(D_b') det(Dhat_b),
with Dhat_b the Schur complement of D_b with respect to its sub-blocks.  With
one level of recursion the hierarchy of acceptance steps (Eq. 4step) is
    0) update the active links (defined by the smallest blocks b'),
    1) accept per sub-block b' with det(D_b'^dag D_b') ratios,
    2) accept per block b with det(Dhat_b^dag Dhat_b) ratios,
    3) accept globally with the Schur complement of the blocks b.
Step 2 is treated stochastically like the global step (Sec. 4): for every
block b, M_b = Dhat_b'^{-1} Dhat_b and ln r_b = -(|M_b eta_b|^2 - |eta_b|^2),
eta_b complex Gaussian on the sites of the black sub-blocks of b.  All blocks
are handled at once: with D1 = sum_b D_b (hops that leave a block b dropped)
and D2 = sum_b' D_b' (hops that leave a sub-block dropped), D1 = D2 + K with
K the hops that cross a sub-block face inside a block; A, E are D2 on the
black / white sub-blocks, B and C the parts of K from white to black and
from black to white.  The delta form of the global step carries over block
by block:
    s = B'E'^{-1}C' eta - A'A^{-1}BE^{-1}C eta,   delta = [D1'^{-1} (s, 0)]_black,
    ln r_b = -sum_{x in b} (2 Re<eta, delta>_x + |delta|_x^2).
Readings (the paper gives no more detail): the sub-blocks tile every block
with an even number of sub-blocks per direction, so the checkerboard of the
sub-blocks inside a block is the global one; the active links are those of
the sub-block decomposition; the proposal/filter iterations repeat steps
0-2 and the global step follows once; noise of step 2 uses purpose 4 and its
uniforms purpose 8 (element = block id).
"""
import numpy as np

from . import accept, dirac, estimator, heatbath, rng
from .geometry import Lattice
from .interp import interpolate
from .solvers import cgnr, norm2, vdot

PURPOSE_BLOCK_SCHUR_NOISE = 4
PURPOSE_BLOCK_SCHUR_ACCEPT = 8


class TwoLevel:
    """Blocks of extent `block`, each split into sub-blocks of extent
    `sub_block`; the active links are those of the sub-blocks."""

    def __init__(self, dims, block, sub_block, active_mode="auto"):
        for b1, b2 in zip(block, sub_block):
            if b1 % b2 or (b1 // b2) % 2:
                raise ValueError("sub-blocks must tile every block with an even number per direction")
        self.lat2 = Lattice(dims, sub_block, active_mode=active_mode)
        self.lat1 = Lattice(dims, block)
        # the active set of the hierarchy is that of the smallest blocks
        self.lat1.active = self.lat2.active.copy()
        self.lat1.active_mode = self.lat2.active_mode
        self.active = self.lat2.active


class Pieces2:
    """A, B, C, E of the sub-block decomposition inside every block, and the
    two Dirichlet operators D1 (blocks) and D2 (sub-blocks), for one field."""

    def __init__(self, U, tl, kappa, tol=1e-14):
        self.U, self.tl, self.kappa, self.tol = U, tl, kappa, tol
        self.black = (tl.lat2.colour == 0)[:, None, None]

    def D1(self, v):
        return dirac.apply_D_dirichlet(self.U, v, self.tl.lat1, self.kappa)

    def D2(self, v):
        return dirac.apply_D_dirichlet(self.U, v, self.tl.lat2, self.kappa)

    def K(self, v):
        # hops across a sub-block face that stay inside a block
        return (dirac.apply_D_inter(self.U, v, self.tl.lat2, self.kappa)
                - dirac.apply_D_inter(self.U, v, self.tl.lat1, self.kappa))

    def _solve(self, op, v):
        opd = lambda w: dirac.apply_gamma5(op(dirac.apply_gamma5(w)))
        x, it, res = cgnr(op, opd, v, tol=self.tol)
        return x

    def D2_solve(self, v):
        return self._solve(self.D2, v)

    def D1_solve(self, v):
        return self._solve(self.D1, v)

    def C(self, v):   # black sub-blocks -> white sub-blocks
        return np.where(self.black, 0, self.K(np.where(self.black, v, 0)))

    def B(self, v):   # white -> black
        return np.where(self.black, self.K(np.where(self.black, 0, v)), 0)


def block_schur_noise(tl, factor, seed, ctr, colour_mask=3):
    """eta on the black sub-block sites of the blocks of colour_mask."""
    lat1, lat2 = tl.lat1, tl.lat2
    sel = (lat2.colour == 0) & np.isin(lat1.colour, [c for c in (0, 1) if colour_mask >> c & 1])
    eta = np.zeros((lat1.V, 4, 3), dtype=np.complex128)
    sites = np.nonzero(sel)[0]
    eta[sites] = rng.spinor_noise(sites, PURPOSE_BLOCK_SCHUR_NOISE, factor, seed, ctr)
    return eta


def block_schur_delta(U, Up, eta, tl, kappa, tol=1e-14):
    """delta = [D1'^{-1} (s, 0)]_black for noise eta (zero off black sub-blocks)."""
    P = Pieces2(U, tl, kappa, tol)
    Pp = Pieces2(Up, tl, kappa, tol)
    v = P.B(P.D2_solve(P.C(eta)))
    a = P.D2_solve(v)
    vp = Pp.B(Pp.D2_solve(Pp.C(eta)))
    s = np.where(P.black, vp - Pp.D2(a), 0)
    y = Pp.D1_solve(s)
    return np.where(P.black, y, 0)


def block_schur_ln_ratios(U, Up, tl, kappa, n, seed, ctr, colour_mask=3, tol=1e-14):
    """Per-block ln r_b of step 2, summed over n interpolation factors (one
    eta per factor); blocks outside colour_mask get 0."""
    lat1 = tl.lat1
    out = np.zeros(lat1.nblocks)
    for i in range(n):
        Ui = interpolate(U, Up, i / n, tl.active)
        Uj = interpolate(U, Up, (i + 1) / n, tl.active)
        eta = block_schur_noise(tl, i, seed, ctr, colour_mask)
        d = block_schur_delta(Ui, Uj, eta, tl, kappa, tol)
        per_site = -(2.0 * np.sum(np.conj(eta) * d, axis=(1, 2)).real + np.sum(np.abs(d) ** 2, axis=(1, 2)))
        out += np.bincount(lat1.block_id, weights=per_site, minlength=lat1.nblocks)
    sel = np.isin(lat1.block_colour, [c for c in (0, 1) if colour_mask >> c & 1])
    out[~sel] = 0.0
    return out


# -------------------------------------------------------------- dense forms
def dense_block_schur(U, tl, kappa, blk):
    """Dhat_b = 1 - A^{-1} B E^{-1} C of block blk, from D_b built directly;
    rows/columns: the black-sub-block sites of blk in local order."""
    lat1, lat2 = tl.lat1, tl.lat2
    sites = lat1.block_sites_of(blk)
    Db = dirac.dense_dirichlet_block(U, lat1, kappa, blk)
    black = lat2.colour[sites] == 0
    ib = dirac.component_index(np.nonzero(black)[0])
    iw = dirac.component_index(np.nonzero(~black)[0])
    A = Db[np.ix_(ib, ib)]
    B = Db[np.ix_(ib, iw)]
    C = Db[np.ix_(iw, ib)]
    E = Db[np.ix_(iw, iw)]
    return np.eye(len(ib)) - np.linalg.solve(A, B @ np.linalg.solve(E, C))


def block_schur_ln_factor_dense(U, Up, eta, tl, kappa, blk):
    """-(|M_b eta_b|^2 - |eta_b|^2) for block blk, M_b = Dhat_b'^{-1} Dhat_b."""
    sites = tl.lat1.block_sites_of(blk)
    black_sites = sites[tl.lat2.colour[sites] == 0]
    e = eta[black_sites].reshape(-1)
    Me = np.linalg.solve(dense_block_schur(Up, tl, kappa, blk), dense_block_schur(U, tl, kappa, blk) @ e)
    return -(norm2(Me) - norm2(e))


def block_schur_ln_ratios_exact(U, Up, tl, kappa, colour_mask=3):
    """2 (ln|det Dhat_b'| - ln|det Dhat_b|) per block, dense LU."""
    lat1 = tl.lat1
    out = np.zeros(lat1.nblocks)
    for blk in range(lat1.nblocks):
        if not (colour_mask >> int(lat1.block_colour[blk]) & 1):
            continue
        out[blk] = 2.0 * (dirac.logabsdet(dense_block_schur(Up, tl, kappa, blk))
                          - dirac.logabsdet(dense_block_schur(U, tl, kappa, blk)))
    return out


# ------------------------------------------------------------------ chain
def block_schur_accept(ln_rb, seed, ctr, colour_mask, block_colour):
    nb = len(ln_rb)
    u = rng.accept_uniform(np.arange(nb, dtype=np.uint64), PURPOSE_BLOCK_SCHUR_ACCEPT, seed, ctr)
    acc = accept.accept_decision(np.asarray(ln_rb), u)
    sel = np.isin(block_colour, [c for c in (0, 1) if colour_mask >> c & 1])
    return np.where(sel, acc, True), np.log(u)


def recursive_step(U, tl, kappa, beta, n_inner, n_sub, n_block, n_global, seed, step, n_or=0, tol=1e-14):
    """One global step of the hierarchy with one level of recursion (Eq. 4step
    steps 0-3).  Counters as in the plain chain: step << 20 | iteration << 4
    for steps 0-2 of an iteration, step << 20 | n_inner << 4 for step 3."""
    from .chain import counter
    lat1, lat2 = tl.lat1, tl.lat2
    U0 = np.array(U, copy=True)
    Ucur = np.array(U, copy=True)
    rec = {"sub": [], "block": [], "ln_global": None, "accept": None, "ln_u": None}
    for it in range(n_inner):
        ctr = counter(step, it, 0)
        Up, _ = heatbath.gauge_update(Ucur, lat2, beta, 1, n_or, seed, ctr, colour_mask=3)
        ln_s = estimator.block_ln_ratios(Ucur, Up, lat2, kappa, n_sub, seed, ctr, colour_mask=3, tol=tol)
        acc_s, lu_s = accept.block_accept(ln_s, seed, ctr, 3, lat2.block_colour)
        Up = accept.restore_rejected_blocks(Up, Ucur, lat2, acc_s)
        rec["sub"].append((ln_s, acc_s, lu_s))
        ln_b = block_schur_ln_ratios(Ucur, Up, tl, kappa, n_block, seed, ctr, colour_mask=3, tol=tol)
        acc_b, lu_b = block_schur_accept(ln_b, seed, ctr, 3, lat1.block_colour)
        rec["block"].append((ln_b, acc_b, lu_b))
        Ucur = accept.restore_rejected_blocks(Up, Ucur, lat1, acc_b)
    ctr = counter(step, n_inner, 0)
    ln = estimator.det_ratio_estimate(U0, Ucur, lat1, kappa, n_global, seed, ctr, tol=tol)
    ok, lu = accept.global_accept(float(np.sum(ln)), seed, ctr)
    rec.update(ln_global=ln, accept=ok, ln_u=lu)
    return (Ucur if ok else U0), rec
