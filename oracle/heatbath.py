"""Wilson plaquette action, heat-bath and over-relaxation on active links (oracle).

Paper Eq. 4step step 0 (the proposal: the active links of every block are
updated by a pure-gauge algorithm such as heat-bath and over-relaxation),
with P_0 ~ exp(-S_G) and the Wilson plaquette action (Sec. 5):  S_G = beta * sum_P (1 - Re tr U_P / 3).

The heat-bath is Cabibbo-Marinari: for each link the SU(2) subgroups
(0,1), (1,2), (0,2) are visited in that order (the order is a reading; the
paper fixes none).  For subgroup (i,j) with staple sum A (six staples) and
W = U A, the 2x2 block w of W is reduced to its quaternion part
k*V (V in SU(2)); the new subgroup element is R = X V^dag with X drawn from
dP(X) ~ exp(alpha * x0) dX_Haar, alpha = 2 beta k / 3.  x0 comes from the
Kennedy-Pendleton sampler (at most 64 tries; after 64 rejections the
subgroup is left unchanged), the direction of (x1, x2, x3) is uniform.
Update: U <- R_emb U.  Over-relaxation uses R = (V^dag)^2, which keeps
Re tr(U A) fixed.

Links are swept direction by direction, and within a direction by site
parity (even sites first); links of one direction and one site parity share
no plaquette, so each such group is updated at once.  In "intra" mode the
sweep is restricted to the selected block colour(s).

Random numbers: Philox stream, purpose 3, element = canonical link index
4*s + a, sub = sweep << 16 | subgroup << 12 | draw; try t uses draws 2t and
2t+1 (uniforms u1..u4), the direction uses draw 200 (u5, u6).
SU(2) parametrisation: [[a0 + i a3, a2 + i a1], [-a2 + i a1, a0 - i a3]].
"""
import numpy as np

from . import rng

SUBGROUPS = ((0, 1), (1, 2), (0, 2))
KP_MAX_TRIES = 64
DIRECTION_DRAW = 200


def dagger(m):
    return np.conj(np.swapaxes(m, -1, -2))


def staple_sum(U, lat, sites, a):
    """Sum of the six staples A of link (s, a) so that U_a(s) A closes the
    plaquettes: A = sum_b [U_b(s+a) U_a(s+b)^dag U_b(s)^dag
                           + U_b(s+a-b)^dag U_a(s-b)^dag U_b(s-b)]."""
    A = np.zeros((len(sites), 3, 3), dtype=np.complex128)
    sa = lat.fwd[sites, a]
    for b in range(4):
        if b == a:
            continue
        sb = lat.fwd[sites, b]
        A += U[sa, b] @ dagger(U[sb, a]) @ dagger(U[sites, b])
        smb = lat.bwd[sites, b]
        samb = lat.bwd[sa, b]
        A += dagger(U[samb, b]) @ dagger(U[smb, a]) @ U[smb, b]
    return A


def plaquette_mean(U, lat):
    """<Re tr U_P / 3> over all 6V plaquettes."""
    tot = 0.0
    for a in range(4):
        for b in range(a + 1, 4):
            s = np.arange(lat.V)
            P = U[s, a] @ U[lat.fwd[s, a], b] @ dagger(U[lat.fwd[s, b], a]) @ dagger(U[s, b])
            tot += np.trace(P, axis1=1, axis2=2).real.sum()
    return tot / (3.0 * 6 * lat.V)


def wilson_action(U, lat, beta):
    return beta * 6 * lat.V * (1.0 - plaquette_mean(U, lat))


def quaternion_of(w):
    """SU(2)-proportional part of 2x2 blocks w: returns (a0, a1, a2, a3)."""
    a0 = 0.5 * (w[:, 0, 0] + w[:, 1, 1]).real
    a3 = 0.5 * (w[:, 0, 0] - w[:, 1, 1]).imag
    a2 = 0.5 * (w[:, 0, 1] - w[:, 1, 0]).real
    a1 = 0.5 * (w[:, 0, 1] + w[:, 1, 0]).imag
    return a0, a1, a2, a3


def su2_matrix(a0, a1, a2, a3):
    m = np.empty((len(a0), 2, 2), dtype=np.complex128)
    m[:, 0, 0] = a0 + 1j * a3
    m[:, 0, 1] = a2 + 1j * a1
    m[:, 1, 0] = -a2 + 1j * a1
    m[:, 1, 1] = a0 - 1j * a3
    return m


def kp_sample_x0(alpha, elements, sub_base, seed, ctr):
    """Kennedy-Pendleton: x0 with density ~ sqrt(1 - x0^2) exp(alpha x0).

    Returns (x0, ok); ok is False where all 64 tries were rejected."""
    n = len(alpha)
    x0 = np.ones(n)
    ok = np.zeros(n, dtype=bool)
    for t in range(KP_MAX_TRIES):
        todo = ~ok
        if not np.any(todo):
            break
        el = elements[todo]
        u1, u2 = rng.uniform_pair(el, rng.PURPOSE_HEATBATH, sub_base + 2 * t, seed, ctr)
        u3, u4 = rng.uniform_pair(el, rng.PURPOSE_HEATBATH, sub_base + 2 * t + 1, seed, ctr)
        c = np.cos(2.0 * np.pi * u2)
        lam2 = -(np.log(u1) + c * c * np.log(u3)) / (2.0 * alpha[todo])
        acc = u4 * u4 <= 1.0 - lam2
        idx = np.nonzero(todo)[0][acc]
        x0[idx] = 1.0 - 2.0 * lam2[acc]
        ok[idx] = True
    return x0, ok


def heatbath_group(U, lat, sites, a, beta, sweep, seed, ctr, overrelax=False):
    """Update the links (s, a), s in sites (independent group), in place.

    Returns the number of subgroup updates left unchanged by the KP cap."""
    elements = (4 * sites + a).astype(np.uint64)
    fails = 0
    A = staple_sum(U, lat, sites, a)
    for sg, (i, j) in enumerate(SUBGROUPS):
        Wm = U[sites, a] @ A
        w = Wm[:, [i, j]][:, :, [i, j]]
        a0, a1, a2, a3 = quaternion_of(w)
        k = np.sqrt(a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3)
        good = k > 1e-300
        ks = np.where(good, k, 1.0)
        Vm = su2_matrix(a0 / ks, a1 / ks, a2 / ks, a3 / ks)
        if overrelax:
            R = dagger(Vm) @ dagger(Vm)
            upd = good
        else:
            sub_base = (sweep << 16) | (sg << 12)
            alpha = 2.0 * beta * ks / 3.0
            x0, ok = kp_sample_x0(alpha, elements, sub_base, seed, ctr)
            fails += int(np.sum(~ok & good))
            u5, u6 = rng.uniform_pair(elements, rng.PURPOSE_HEATBATH, sub_base + DIRECTION_DRAW, seed, ctr)
            r = np.sqrt(np.maximum(0.0, 1.0 - x0 * x0))
            cth = 2.0 * u5 - 1.0
            sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
            phi = 2.0 * np.pi * u6
            X = su2_matrix(x0, r * sth * np.cos(phi), r * sth * np.sin(phi), r * cth)
            R = X @ dagger(Vm)
            upd = good & ok
        rows = U[sites, a][:, [i, j], :]
        new = R @ rows
        Ua = U[sites, a]
        Ua[upd, i, :] = new[upd, 0, :]
        Ua[upd, j, :] = new[upd, 1, :]
        U[sites, a] = Ua
    return fails


def gauge_update(U, lat, beta, n_hb, n_or, seed, ctr, colour_mask=3, active=None):
    """n_hb heat-bath sweeps, each followed by n_or over-relaxation sweeps, on
    the active links of the selected block colours.  Returns (U', fails)."""
    U = np.array(U, copy=True)
    act = lat.active if active is None else active
    link_colour = lat.colour
    fails = 0
    for sweep in range(n_hb):
        for kind in [False] + [True] * n_or:
            for a in range(4):
                for par in (0, 1):
                    sel = act[:, a] & (lat.parity == par) & np.isin(link_colour, [c for c in (0, 1) if colour_mask >> c & 1])
                    sites = np.nonzero(sel)[0]
                    if len(sites):
                        fails += heatbath_group(U, lat, sites, a, beta, sweep, seed, ctr, overrelax=kind)
    return U, fails
