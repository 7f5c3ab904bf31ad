"""Stochastic determinant-ratio estimates (oracle).

Paper Sec. 4: with M = Dhat'^{-1} Dhat the exact acceptance step
min{1, det(M^dag M)} is replaced by min{1, exp(-eta^dag (M^dag M - 1) eta)},
a fresh complex Gaussian eta for every step; the expectation over eta of
exp(-eta^dag (A - 1) eta) is 1/det A.  With the interpolation factorisation
(Eq. param) the ratio is the product over N factors M_i = Dhat[U_{i+1}]^{-1}
Dhat[U_i], each with its own noise vector; the log of the estimate is
    ln r = sum_i -(|M_i eta_i|^2 - |eta_i|^2).

Two forms are computed here:
  * ``ln_factor_dense``: the definition, with dense D, Dhat and M (small
    lattices only);
  * ``ln_factor_delta``: the same number through delta = (M - 1) eta, so
    ln r_i = -(2 Re<eta, delta> + |delta|^2).  Using
    Dhat'^{-1} = (D'^{-1})_bb A' (block inverse of Eq. domdec) and
    A'(Dhat - Dhat') = B' E'^{-1} C' - A' A^{-1} B E^{-1} C,
    delta = [D'^{-1} (s, 0)]_black with s = B'E'^{-1}C' eta - A'A^{-1}BE^{-1}C eta.
    The difference of two O(V) norms never has to be formed, so the result
    keeps its absolute accuracy on large lattices.
Block filter (Eq. 4step step 1, Sec. 5): the same with M_b = D_b'^{-1} D_b per
block, delta_b = D_b'^{-1}(D_b - D_b') eta_b; the exact mode uses
ln r_b = ln det(D_b'^dag D_b') - ln det(D_b^dag D_b) = 2(ln|det D_b'| - ln|det D_b|).
"""
import numpy as np

from . import dirac, rng
from .interp import interpolate
from .solvers import cgnr, norm2, vdot


# -------------------------------------------------------------- dense forms
def ln_factor_dense(U, Up, eta_black, lat, kappa):
    """-(|M eta|^2 - |eta|^2), M = Dhat[Up]^{-1} Dhat[U], eta in block order."""
    Dh = dirac.dense_schur(dirac.dense_D(U, lat, kappa), lat)
    Dhp = dirac.dense_schur(dirac.dense_D(Up, lat, kappa), lat)
    e = eta_black.reshape(-1)
    Me = np.linalg.solve(Dhp, Dh @ e)
    return -(norm2(Me) - norm2(e))


def exact_ln_ratio_schur(U, Up, lat, kappa):
    """ln det(M^dag M) = 2 (ln|det Dhat| - ln|det Dhat'|), dense."""
    Dh = dirac.dense_schur(dirac.dense_D(U, lat, kappa), lat)
    Dhp = dirac.dense_schur(dirac.dense_D(Up, lat, kappa), lat)
    return 2.0 * (dirac.logabsdet(Dh) - dirac.logabsdet(Dhp))


# ------------------------------------------------------- operator pieces
class Pieces:
    """Apply the pieces A, B, C, E of Eq. domdec for one gauge field."""

    def __init__(self, U, lat, kappa, tol=1e-14):
        self.U, self.lat, self.kappa, self.tol = U, lat, kappa, tol
        self.black = (lat.colour == 0)[:, None, None]
        self.iters = 0

    def inter(self, v):
        return dirac.apply_D_inter(self.U, v, self.lat, self.kappa)

    def dirichlet(self, v):
        return dirac.apply_D_dirichlet(self.U, v, self.lat, self.kappa)

    def dirichlet_dag(self, v):
        # adjoint of the block-diagonal operator: gamma5 D_b gamma5
        return dirac.apply_gamma5(self.dirichlet(dirac.apply_gamma5(v)))

    def dirichlet_solve(self, v):
        """(D_bb + D_ww)^{-1} v: all block solves of the colour(s) v lives on."""
        x, it, res = cgnr(self.dirichlet, self.dirichlet_dag, v, tol=self.tol)
        self.iters += it
        return x

    def C(self, v):   # black -> white
        return np.where(self.black, 0, self.inter(np.where(self.black, v, 0)))

    def B(self, v):   # white -> black
        return np.where(self.black, self.inter(np.where(self.black, 0, v)), 0)


def full_solve(U, b, lat, kappa, tol=1e-14):
    A = lambda v: dirac.apply_D(U, v, lat, kappa)
    Ad = lambda v: dirac.apply_gamma5(dirac.apply_D(U, dirac.apply_gamma5(v), lat, kappa))
    return cgnr(A, Ad, b, tol=tol)


def delta_source(U, Up, eta_full, lat, kappa, tol=1e-14):
    """s = B'E'^{-1}C' eta - A'A^{-1}BE^{-1}C eta (black sites, full-lattice array)."""
    P = Pieces(U, lat, kappa, tol)
    Pp = Pieces(Up, lat, kappa, tol)
    v = P.B(P.dirichlet_solve(P.C(eta_full)))
    a = P.dirichlet_solve(v)
    vp = Pp.B(Pp.dirichlet_solve(Pp.C(eta_full)))
    s = vp - Pp.dirichlet(a)
    return np.where(P.black, s, 0)


def ln_factor_delta(U, Up, eta_full, lat, kappa, tol=1e-14):
    """ln r_i in the delta form; eta_full is zero on white sites."""
    s = delta_source(U, Up, eta_full, lat, kappa, tol)
    y, it, res = full_solve(Up, s, lat, kappa, tol)
    black = (lat.colour == 0)[:, None, None]
    d = np.where(black, y, 0)
    return -(2.0 * vdot(eta_full, d).real + norm2(d))


def global_noise(lat, factor, seed, ctr):
    """eta_i on the black sites (zero on white), full-lattice array."""
    eta = np.zeros((lat.V, 4, 3), dtype=np.complex128)
    sites = lat.black_sites()
    eta[sites] = rng.spinor_noise(sites, rng.PURPOSE_GLOBAL_NOISE, factor, seed, ctr)
    return eta


def det_ratio_estimate(U, Up, lat, kappa, n, seed, ctr, mode="factors", tol=1e-14, dense=False, interp_mask=None):
    """Per-factor ln r_i of the global (Schur complement) step, length n.

    mode "factors": factor i uses U_i, U_{i+1} of the n-step interpolation and
    its own eta_i.  mode "replicas": every factor uses the pair (U, U') with
    its own eta_i (the variance measurement of Sec. 5).  interp_mask: the
    links the interpolation runs over (default: the active links; after a
    relative gauge fixing: every link that differs).
    """
    mask = lat.active if interp_mask is None else interp_mask
    out = np.empty(n)
    for i in range(n):
        if mode == "factors":
            Ui = interpolate(U, Up, i / n, mask)
            Uj = interpolate(U, Up, (i + 1) / n, mask)
        else:
            Ui, Uj = U, Up
        eta = global_noise(lat, i, seed, ctr)
        if dense:
            out[i] = ln_factor_dense(Ui, Uj, eta[lat.black_sites()], lat, kappa)
        else:
            out[i] = ln_factor_delta(Ui, Uj, eta, lat, kappa, tol)
    return out


# -------------------------------------------------------------- block filter
def block_noise(lat, factor, seed, ctr):
    sites = np.arange(lat.V)
    return rng.spinor_noise(sites, rng.PURPOSE_BLOCK_NOISE, factor, seed, ctr)


def block_ln_ratios(U, Up, lat, kappa, n, seed, ctr, colour_mask=3, tol=1e-14):
    """Per-block ln r_b summed over n interpolation factors (stochastic).

    Blocks of colours outside colour_mask get 0.
    """
    sel = np.isin(lat.colour, [c for c in (0, 1) if colour_mask >> c & 1])
    out = np.zeros(lat.nblocks)
    for i in range(n):
        Ui = interpolate(U, Up, i / n, lat.active)
        Uj = interpolate(U, Up, (i + 1) / n, lat.active)
        eta = np.where(sel[:, None, None], block_noise(lat, i, seed, ctr), 0)
        Pi = Pieces(Ui, lat, kappa, tol)
        Pj = Pieces(Uj, lat, kappa, tol)
        src = Pi.dirichlet(eta) - Pj.dirichlet(eta)
        d = Pj.dirichlet_solve(src)
        per_site = -(2.0 * np.sum(np.conj(eta) * d, axis=(1, 2)).real + np.sum(np.abs(d) ** 2, axis=(1, 2)))
        out += np.bincount(lat.block_id, weights=per_site, minlength=lat.nblocks)
    return out


def block_ln_ratios_exact(U, Up, lat, kappa, colour_mask=3):
    """2 (ln|det D_b'| - ln|det D_b|) per block, dense LU."""
    out = np.zeros(lat.nblocks)
    for blk in range(lat.nblocks):
        if not (colour_mask >> int(lat.block_colour[blk]) & 1):
            continue
        out[blk] = 2.0 * (dirac.logabsdet(dirac.dense_dirichlet_block(Up, lat, kappa, blk))
                          - dirac.logabsdet(dirac.dense_dirichlet_block(U, lat, kappa, blk)))
    return out
