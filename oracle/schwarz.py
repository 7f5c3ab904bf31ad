"""Schwarz alternating procedure and flexible GCR (oracle).

The block decomposition of Sec. 3 (black/white checkerboard of blocks,
Eq. domdec) is the one of Luscher's Schwarz-preconditioned solver, which the
paper names as the origin of domain decomposition for lattice QCD.  Used as
a preconditioner of the global solve it gives:

Multiplicative Schwarz (SAP), ncy cycles on D z = rho from z = 0:
    for every cycle, for colour c = black, then white:
        r = rho - D z                       (the current residual)
        z_b += D_b^{-1} r_b   for every block b of colour c
with D_b the Dirichlet block operator (hops that leave the block dropped).
The blocks of one colour share no hop, so their solves are independent.
With exact block solves one cycle is the block Gauss-Seidel step of
D = [[A, B], [C, E]] (black sites first):  z = [[A, 0], [C, E]]^{-1} rho,
and cycle k + 1 adds that step applied to the residual of cycle k.

Flexible GCR (the generalised conjugate residual method with a
preconditioner that may change from one iteration to the next): from x and
r = b - A x, for k = 0, 1, ...:
    z_k = M_k(r), w_k = A z_k,
    w_k and z_k orthogonalised against the earlier w_j (modified
    Gram-Schmidt, the same coefficients applied to z), then w_k scaled to
    unit norm (and z_k with it),
    alpha = <w_k, r>, x += alpha z_k, r -= alpha w_k,
restarting after nkv directions with the recursively updated r (the true
residual is recomputed once at every restart).  The residual norm never
grows (each step minimises |r| over the directions kept).

The block solves are exact here: dense LU factorisations of every D_b,
computed once per gauge field.  Plain numpy/scipy FP64.
"""
import numpy as np
import scipy.linalg

from . import dirac
from .solvers import norm2, vdot


class BlockSolver:
    """Exact Dirichlet block solves for one gauge field: an LU factorisation
    of every D_b (dense), applied block by block."""

    def __init__(self, U, lat, kappa):
        self.lat = lat
        self.sites = [lat.block_sites_of(b) for b in range(lat.nblocks)]
        self.lu = [scipy.linalg.lu_factor(dirac.dense_dirichlet_block(U, lat, kappa, b))
                   for b in range(lat.nblocks)]

    def solve_colour(self, r, colour):
        """D_b^{-1} r_b on every block b of the given colour, 0 elsewhere."""
        out = np.zeros_like(r)
        for b in range(self.lat.nblocks):
            if self.lat.block_colour[b] != colour:
                continue
            s = self.sites[b]
            out[s] = scipy.linalg.lu_solve(self.lu[b], r[s].reshape(-1)).reshape(len(s), 4, 3)
        return out


def sap(U, lat, kappa, rho, ncy, blocks=None):
    """ncy cycles of the Schwarz alternating procedure on D z = rho from z = 0."""
    blocks = blocks or BlockSolver(U, lat, kappa)
    z = np.zeros_like(rho)
    for _ in range(ncy):
        for colour in (0, 1):
            r = rho - dirac.apply_D(U, z, lat, kappa)
            z = z + blocks.solve_colour(r, colour)
    return z


def fgcr(apply_A, precond, b, tol=1e-12, nkv=8, maxit=1000, history=None):
    """Flexible GCR with restarts after nkv directions.  Returns
    (x, iterations, true relative residual); `history` (a list) collects
    |r| after every iteration."""
    bn = np.sqrt(norm2(b))
    x = np.zeros_like(b)
    if bn == 0.0:
        return x, 0, 0.0
    r = np.array(b, copy=True)
    it = 0
    while it < maxit:
        zs, ws = [], []
        for _ in range(nkv):
            z = precond(r)
            w = apply_A(z)
            for zj, wj in zip(zs, ws):
                c = vdot(wj, w)
                w = w - c * wj
                z = z - c * zj
            nw = np.sqrt(norm2(w))
            w, z = w / nw, z / nw
            alpha = vdot(w, r)
            x = x + alpha * z
            r = r - alpha * w
            zs.append(z)
            ws.append(w)
            it += 1
            rn = np.sqrt(norm2(r))
            if history is not None:
                history.append(rn)
            if rn <= tol * bn or it >= maxit:
                break
        r = b - apply_A(x)           # restart from the true residual
        if np.sqrt(norm2(r)) <= tol * bn:
            break
    return x, it, float(np.sqrt(norm2(b - apply_A(x))) / bn)


def sap_gcr_solve(U, lat, kappa, b, tol=1e-12, ncy=2, nkv=8, maxit=1000):
    """D x = b by flexible GCR preconditioned with ncy SAP cycles (exact
    block solves).  Returns (x, GCR iterations, true relative residual)."""
    blocks = BlockSolver(U, lat, kappa)
    A = lambda v: dirac.apply_D(U, v, lat, kappa)
    M = lambda r: sap(U, lat, kappa, r, ncy, blocks)
    return fgcr(A, M, b, tol=tol, nkv=nkv, maxit=maxit)
