"""Uniforms and complex Gaussian noise from Philox4x32-10 (oracle).

Stream convention (shared by definition with the CUDA path, which implements
the same generator on its own):
  key     = (seed mod 2^32, seed >> 32)
  counter = (element, purpose << 24 | sub, ctr mod 2^32, ctr >> 32)
One Philox call gives two 53-bit uniforms
  u = (k + 1/2) * 2^-53,  k = (w_a << 21) | (w_b >> 11),
from the word pairs (w0, w1) and (w2, w3); u lies strictly inside (0, 1).

Noise (Sec. 4): the estimator E[exp(-eta^dag (A - 1) eta)] = 1/det A needs
the density p(eta) ~ exp(-eta^dag eta), i.e. Re and Im of every component
N(0, 1/2).  The paper does not state the normalisation; this is the one for
which the identity holds.  Box-Muller on the two uniforms of one call:
  eta = sqrt(-ln u1) * (cos(2 pi u2) + i sin(2 pi u2)).
Element index of a spinor component = canonical site * 12 + spin * 3 + colour.
"""
import numpy as np

from .philox import philox4x32_10

PURPOSE_GLOBAL_NOISE = 1
PURPOSE_BLOCK_NOISE = 2
PURPOSE_HEATBATH = 3
PURPOSE_BLOCK_ACCEPT = 5
PURPOSE_GLOBAL_ACCEPT = 6
PURPOSE_USER_NOISE = 7

TWO_M53 = 2.0 ** -53


def _split(v):
    v = int(v)
    return v & 0xFFFFFFFF, (v >> 32) & 0xFFFFFFFF


def raw_words(element, purpose, sub, seed, ctr):
    k0, k1 = _split(seed)
    c2, c3 = _split(ctr)
    c1 = (np.asarray(purpose, dtype=np.uint64) << np.uint64(24)) | (np.asarray(sub, dtype=np.uint64) & np.uint64(0xFFFFFF))
    return philox4x32_10(element, c1, c2, c3, k0, k1)


def words_to_uniform(wa, wb):
    k = (wa.astype(np.uint64) << np.uint64(21)) | (wb.astype(np.uint64) >> np.uint64(11))
    return (k.astype(np.float64) + 0.5) * TWO_M53


def uniform_pair(element, purpose, sub, seed, ctr):
    w0, w1, w2, w3 = raw_words(element, purpose, sub, seed, ctr)
    return words_to_uniform(w0, w1), words_to_uniform(w2, w3)


def gaussian_components(element, purpose, sub, seed, ctr):
    """One complex Gaussian number per element index (N(0,1/2) per part)."""
    u1, u2 = uniform_pair(element, purpose, sub, seed, ctr)
    r = np.sqrt(-np.log(u1))
    ang = 2.0 * np.pi * u2
    return r * np.cos(ang) + 1j * r * np.sin(ang)


def spinor_noise(sites, purpose, sub, seed, ctr):
    """Complex Gaussian spinor on the given canonical sites, shape (n, 4, 3)."""
    sites = np.asarray(sites, dtype=np.uint64)
    el = sites[:, None] * np.uint64(12) + np.arange(12, dtype=np.uint64)[None, :]
    return gaussian_components(el, purpose, sub, seed, ctr).reshape(len(sites), 4, 3)


def accept_uniform(element, purpose, seed, ctr):
    """The uniform u that a Metropolis step compares against (first of the pair)."""
    u1, _ = uniform_pair(np.asarray(element, dtype=np.uint64), purpose, 0, seed, ctr)
    return u1
