"""Relative gauge fixing of a proposal to the current configuration (oracle).

Sec. 4: the variance of the eigenvalue distribution of M^dag M can be reduced
by relative gauge fixing of the old and the proposed link configuration; the
paper does not state the method.  Reading taken here: maximise
    F[g] = sum_{x, a} Re tr( U_a(x)^dag g(x) U'_a(x) g(x + a)^dag )
over site-local SU(3) matrices g, i.e. bring U'^g_a(x) = g(x) U'_a(x) g(x+a)^dag
as close to U as local gauge freedom allows.  Starting from g = 1, a sweep
visits the sites of one parity at a time (sites of one parity share no link,
so their local problems are independent); at site x,
    F = Re tr(g(x) W(x)) + const,
    W(x) = sum_a [ U'_a(x) g(x+a)^dag U_a(x)^dag + (U_a(x-a)^dag g(x-a) U'_a(x-a))^dag ],
which is raised by Cabibbo-Marinari steps over the SU(2) subgroups (0,1),
(1,2), (0,2): with the 2x2 block of g W reduced to k V (V in SU(2)), the
subgroup element R = V^dag maximises it and g(x) <- R g(x).
Because g is site-diagonal, D[U'^g] = G D[U'] G^dag and every block and
Schur complement transforms by a similarity: all determinant ratios of
Eq. 4step are unchanged.  The estimate then uses U'^g, with the
interpolation running over every link that differs from U.
"""
import numpy as np

from . import dirac
from .heatbath import SUBGROUPS, dagger, quaternion_of, su2_matrix


def functional(U, Up, g, lat):
    """F[g] = sum Re tr(U^dag g U' g(x+a)^dag)."""
    tot = 0.0
    for a in range(4):
        M = dagger(U[:, a]) @ g @ Up[:, a] @ dagger(g[lat.fwd[:, a]])
        tot += np.trace(M, axis1=1, axis2=2).real.sum()
    return float(tot)


def local_w(U, Up, g, lat, sites):
    W = np.zeros((len(sites), 3, 3), dtype=np.complex128)
    for a in range(4):
        y = lat.fwd[sites, a]
        W += Up[sites, a] @ dagger(g[y]) @ dagger(U[sites, a])
        z = lat.bwd[sites, a]
        W += dagger(dagger(U[z, a]) @ g[z] @ Up[z, a])
    return W


def maximise(gx, W):
    """One Cabibbo-Marinari pass raising Re tr(g W) for a set of sites."""
    gx = np.array(gx, copy=True)
    for (i, j) in SUBGROUPS:
        M = gx @ W
        w = M[:, [i, j]][:, :, [i, j]]
        a0, a1, a2, a3 = quaternion_of(w)
        k = np.sqrt(a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3)
        good = k > 1e-300
        ks = np.where(good, k, 1.0)
        R = dagger(su2_matrix(a0 / ks, a1 / ks, a2 / ks, a3 / ks))
        rows = gx[:, [i, j], :]
        new = R @ rows
        gx[good, i, :] = new[good, 0, :]
        gx[good, j, :] = new[good, 1, :]
    return gx


def relative_gauge_fix(U, Up, lat, sweeps):
    """Returns (g, U'^g, [F after each sweep]) starting from g = 1."""
    g = np.zeros((lat.V, 3, 3), dtype=np.complex128)
    g[:, 0, 0] = g[:, 1, 1] = g[:, 2, 2] = 1.0
    history = [functional(U, Up, g, lat)]
    for _ in range(sweeps):
        for par in (0, 1):
            sites = np.nonzero(lat.parity == par)[0]
            W = local_w(U, Up, g, lat, sites)
            g[sites] = maximise(g[sites], W)
        history.append(functional(U, Up, g, lat))
    return g, dirac.gauge_transform_links(Up, g, lat), history


def differing_links(U, Up):
    """(V, 4) mask of the links where U and U' differ."""
    return np.any(U != Up, axis=(2, 3))
