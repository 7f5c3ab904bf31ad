"""Interpolated link configurations U_i, i = 0..N (oracle).

Paper Sec. 4, Eq. param: the change U -> U' is split into a sequence with
U_0 = U, U_N = U' and ||U_i - U_{i+1}|| proportional to 1/N.  The path itself
is not specified in the paper.  Reading taken: the SU(3) geodesic
    U_t = U W^t,  W = U^dag U',  t = i/N,
with W^t = V diag(exp(i t theta_j)) V^{-1} from the eigen-decomposition of W,
theta_j in (-pi, pi].  For SU(3) the principal phases sum to 0 or +-2 pi; when
the sum is +2 pi the largest phase is lowered by 2 pi, when it is -2 pi the
smallest is raised by 2 pi, so that det W^t = 1 along the whole path.  The
reversed path (U' -> U) is then the same set of links, as detailed balance
requires.  Links that do not change (W = 1) stay exactly equal.
"""
import numpy as np


def su3_power(W, t):
    """W^t for stacked SU(3) matrices W (shape (n, 3, 3)), with the branch above."""
    W = np.asarray(W)
    lam, vec = np.linalg.eig(W)
    theta = np.angle(lam)
    tot = theta.sum(axis=1)
    hi = tot > np.pi          # sum is +2 pi
    lo = tot < -np.pi         # sum is -2 pi
    if np.any(hi):
        j = np.argmax(theta[hi], axis=1)
        theta[np.nonzero(hi)[0], j] -= 2 * np.pi
    if np.any(lo):
        j = np.argmin(theta[lo], axis=1)
        theta[np.nonzero(lo)[0], j] += 2 * np.pi
    ph = np.exp(1j * t * theta)
    return np.einsum("nik,nk,nkj->nij", vec, ph, np.linalg.inv(vec))


def interpolate(U, Up, t, mask=None):
    """U_t = U (U^dag U')^t on the links where mask is set (all links if None);
    U_0 = U exactly and U_1 = U' exactly."""
    out = np.array(U, copy=True)
    if t == 0:
        return out
    if mask is None:
        mask = np.ones(U.shape[:2], dtype=bool)
    if t == 1:
        out[mask] = Up[mask]
        return out
    a = U[mask]
    b = Up[mask]
    W = np.conj(np.transpose(a, (0, 2, 1))) @ b
    out[mask] = a @ su3_power(W, t)
    return out
