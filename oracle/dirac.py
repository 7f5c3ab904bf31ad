"""Wilson-Dirac operator and its domain-decomposed pieces (oracle, FP64).

Definitions (paper Sec. 3 and 5; the paper names the plain Wilson-Dirac
operator without writing it out, so the standard hopping form is taken):

    D = 1 - kappa * H,
    (H psi)(x) = sum_a [ (1 - gamma_a) U_a(x) psi(x + a) s_f(x, a)
                       + (1 + gamma_a) U_a(x - a)^dag psi(x - a) s_b(x, a) ]

with s_f, s_b = bc_time (-1, antiperiodic) on hops that wrap the time extent
and 1 otherwise; links are periodic.  Spinors have shape (V, 4, 3), links
(V, 4, 3, 3).

Domain decomposition (Eq. domdec, Eq. ddfactor): with sites ordered black
blocks first, D = [[A, B], [C, E]] where A = D_bb and E = D_ww are block
diagonal with the Dirichlet block operators D_b (every hop that leaves the
block dropped), and B = D_bw, C = D_wb hold the hops that cross block faces.
The Schur complement is Dhat = 1 - A^{-1} B E^{-1} C on the black sites.

Even-odd: with sites split by parity, D = [[1, -kappa H_eo], [-kappa H_oe, 1]]
and the even-site Schur complement is Dtilde = 1 - kappa^2 H_eo H_oe.
"""
import numpy as np

from .gamma import GAMMA_AXIS, GAMMA5, ONE4

# hop selectors
ALL, INTRA, INTER = "all", "intra", "inter"


def _hop_allowed(lat, sel, a, forward):
    nb = lat.fwd[:, a] if forward else lat.bwd[:, a]
    if sel == ALL:
        return None
    same = lat.block_id[nb] == lat.block_id
    return same if sel == INTRA else ~same


def hop(U, psi, lat, sel=ALL):
    """H psi (sel = "all"), or its intra-block / inter-block part."""
    out = np.zeros_like(psi)
    for a in range(4):
        g = GAMMA_AXIS[a]
        f = lat.fwd[:, a]
        b = lat.bwd[:, a]
        # forward hop: (1 - gamma_a) U_a(x) psi(x + a)
        up = np.einsum("xij,xsj->xsi", U[:, a], psi[f])
        tf = np.einsum("st,xti->xsi", ONE4 - g, up) * lat.sign_fwd[:, a, None, None]
        # backward hop: (1 + gamma_a) U_a(x - a)^dag psi(x - a)
        dn = np.einsum("xji,xsj->xsi", np.conj(U[b, a]), psi[b])
        tb = np.einsum("st,xti->xsi", ONE4 + g, dn) * lat.sign_bwd[:, a, None, None]
        mf = _hop_allowed(lat, sel, a, True)
        mb = _hop_allowed(lat, sel, a, False)
        if mf is not None:
            tf = tf * mf[:, None, None]
            tb = tb * mb[:, None, None]
        out += tf + tb
    return out


def apply_D(U, psi, lat, kappa):
    """D psi = psi - kappa H psi (whole lattice)."""
    return psi - kappa * hop(U, psi, lat, ALL)


def apply_D_dirichlet(U, psi, lat, kappa):
    """(D_bb + D_ww) psi: every block's Dirichlet operator D_b at once."""
    return psi - kappa * hop(U, psi, lat, INTRA)


def apply_D_inter(U, psi, lat, kappa):
    """(D_bw + D_wb) psi = -kappa * (hops crossing block faces) psi."""
    return -kappa * hop(U, psi, lat, INTER)


def apply_gamma5(psi):
    return np.einsum("st,...ti->...si", GAMMA5, psi)


def apply_Ddag(U, psi, lat, kappa):
    """D^dag psi via gamma5-hermiticity is NOT used here: D^dag is taken
    as the adjoint of the explicit stencil, term by term."""
    out = np.array(psi, copy=True)
    for a in range(4):
        g = GAMMA_AXIS[a]
        f = lat.fwd[:, a]
        b = lat.bwd[:, a]
        # adjoint of the forward term of site b: (1 - g)^dag U_a(x - a)^dag psi(x - a)
        dn = np.einsum("xji,xsj->xsi", np.conj(U[b, a]), psi[b])
        t1 = np.einsum("ts,xti->xsi", np.conj(ONE4 - g), dn) * lat.sign_fwd[b, a, None, None]
        # adjoint of the backward term of site f: (1 + g)^dag U_a(x) psi(x + a)
        up = np.einsum("xij,xsj->xsi", U[:, a], psi[f])
        t2 = np.einsum("ts,xti->xsi", np.conj(ONE4 + g), up) * lat.sign_bwd[f, a, None, None]
        out -= kappa * (t1 + t2)
    return out


# --------------------------------------------------------------- dense forms
def dense_D(U, lat, kappa):
    """D as a dense (12V x 12V) matrix, index = site*12 + spin*3 + colour.

    Built entry by entry from the definition (not by applying the stencil to
    unit vectors), so it is an independent restatement of the operator.
    """
    n = 12 * lat.V
    D = np.eye(n, dtype=np.complex128)
    for x in range(lat.V):
        for a in range(4):
            g = GAMMA_AXIS[a]
            y = lat.fwd[x, a]
            D[12 * x:12 * x + 12, 12 * y:12 * y + 12] -= kappa * lat.sign_fwd[x, a] * np.kron(ONE4 - g, U[x, a])
            y = lat.bwd[x, a]
            D[12 * x:12 * x + 12, 12 * y:12 * y + 12] -= kappa * lat.sign_bwd[x, a] * np.kron(ONE4 + g, np.conj(U[y, a]).T)
    return D


def dense_dirichlet_block(U, lat, kappa, blk):
    """D_b of Eq. domdec built directly: hops between sites of block blk only,
    sites in local lexicographic order (the Dirichlet boundary condition)."""
    sites = lat.block_sites_of(blk)
    pos = {int(s): k for k, s in enumerate(sites)}
    n = 12 * len(sites)
    D = np.eye(n, dtype=np.complex128)
    for k, x in enumerate(sites):
        for a in range(4):
            g = GAMMA_AXIS[a]
            y = int(lat.fwd[x, a])
            if y in pos:
                j = pos[y]
                D[12 * k:12 * k + 12, 12 * j:12 * j + 12] -= kappa * lat.sign_fwd[x, a] * np.kron(ONE4 - g, U[x, a])
            y = int(lat.bwd[x, a])
            if y in pos:
                j = pos[y]
                D[12 * k:12 * k + 12, 12 * j:12 * j + 12] -= kappa * lat.sign_bwd[x, a] * np.kron(ONE4 + g, np.conj(U[y, a]).T)
    return D


def component_index(sites):
    """Flat component indices (site*12 + k) of the given sites, in order."""
    sites = np.asarray(sites)
    return (12 * sites[:, None] + np.arange(12)[None, :]).reshape(-1)


def dd_blocks(Dfull, lat):
    """Split a dense D into A = D_bb, B = D_bw, C = D_wb, E = D_ww (block order)."""
    idx = component_index(lat.dd_order)
    P = Dfull[np.ix_(idx, idx)]
    nb = 12 * lat.n_black_sites
    return P[:nb, :nb], P[:nb, nb:], P[nb:, :nb], P[nb:, nb:]


def dense_schur(Dfull, lat):
    """Dhat = 1 - A^{-1} B E^{-1} C on the black sites (Eq. ddfactor)."""
    A, B, C, E = dd_blocks(Dfull, lat)
    return np.eye(A.shape[0]) - np.linalg.solve(A, B @ np.linalg.solve(E, C))


def dense_block_operator(Dfull, lat, blk):
    """D_b: the principal submatrix of D on the sites of block blk (Dirichlet)."""
    idx = component_index(lat.block_sites_of(blk))
    return Dfull[np.ix_(idx, idx)]


def dense_even_odd(Dfull, lat, kappa):
    """Return (H_eo, H_oe, Dtilde) from a dense D, sites of each parity in
    canonical order."""
    ev = component_index(np.nonzero(lat.parity == 0)[0])
    od = component_index(np.nonzero(lat.parity == 1)[0])
    H_eo = -Dfull[np.ix_(ev, od)] / kappa
    H_oe = -Dfull[np.ix_(od, ev)] / kappa
    Dt = np.eye(len(ev)) - kappa * kappa * H_eo @ H_oe
    return H_eo, H_oe, Dt


def logabsdet(M):
    """ln|det M| by LU (numpy/LAPACK slogdet)."""
    sign, ld = np.linalg.slogdet(M)
    return float(ld)


# ------------------------------------------------------------ gauge transform
def gauge_transform_links(U, g, lat):
    """U^g_a(x) = g(x) U_a(x) g(x + a)^dag."""
    out = np.empty_like(U)
    for a in range(4):
        out[:, a] = g @ U[:, a] @ np.conj(np.transpose(g[lat.fwd[:, a]], (0, 2, 1)))
    return out


def gauge_transform_spinor(psi, g):
    return np.einsum("xij,xsj->xsi", g, psi)
