"""Seeded synthetic inputs (gauge fields, gauge transformations, spinors).

This module only synthesises inputs; it holds none of the method's arithmetic
(no Dirac operator, no solver, no estimator, no random stream of the method).
Both the CPU oracle's tests and the CUDA path's tests and benchmark draw their
inputs from here, so the two sides always start from identical bits.

Field conventions (canonical layout, FP64):
  * site index   s = x0 + L0*(x1 + L1*(x2 + L2*x3)), axis 3 is time;
  * gauge field  U[s, a, i, j]  complex128, shape (V, 4, 3, 3): the SU(3) link
                 from site s to s + a-hat (a = lattice axis 0..3);
  * spinor       psi[s, spin, colour] complex128, shape (V, 4, 3).

Gauge links follow the synthetic recipe U = exp(i * eps * H) with
H = sum_{k=1..8} w_k lambda_k, w_k ~ N(0, 1) and lambda_k the Gell-Mann
matrices (so every off-diagonal real and imaginary part of H is N(0, 1)).
The exponential is taken through the Hermitian eigendecomposition, and the
result is re-unitarised (rows 1-2 orthonormalised, row 3 = conj(row1 x row2))
so that every link is in SU(3) to rounding.
"""
import os

import numpy as np

__all__ = ["gell_mann", "random_su3", "random_gauge", "random_spinor",
           "random_gauge_transform", "unit_gauge", "lattice_volume"]


def gell_mann():
    """The eight Gell-Mann matrices, shape (8, 3, 3) complex128."""
    g = np.zeros((8, 3, 3), dtype=np.complex128)
    g[0, 0, 1] = g[0, 1, 0] = 1
    g[1, 0, 1] = -1j
    g[1, 1, 0] = 1j
    g[2, 0, 0] = 1
    g[2, 1, 1] = -1
    g[3, 0, 2] = g[3, 2, 0] = 1
    g[4, 0, 2] = -1j
    g[4, 2, 0] = 1j
    g[5, 1, 2] = g[5, 2, 1] = 1
    g[6, 1, 2] = -1j
    g[6, 2, 1] = 1j
    g[7, 0, 0] = g[7, 1, 1] = 1 / np.sqrt(3)
    g[7, 2, 2] = -2 / np.sqrt(3)
    return g


def lattice_volume(dims):
    v = 1
    for d in dims:
        v *= int(d)
    return v


def _reunitarise(u):
    """Project stacked 3x3 matrices back onto SU(3) (Gram-Schmidt rows 1-2)."""
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def random_su3(shape, eps, rng, chunk=1 << 16):
    """exp(i*eps*H) for H a Gaussian combination of Gell-Mann matrices.

    The Gaussian weights are drawn in one sequential pass (so the result does
    not depend on the chunking); the exponentials run in parallel chunks."""
    from concurrent.futures import ThreadPoolExecutor
    lam = gell_mann()
    n = int(np.prod(shape)) if len(shape) else 1
    w_all = rng.standard_normal((n, 8))
    out = np.empty((n, 3, 3), dtype=np.complex128)

    def work(lo):
        hi = min(n, lo + chunk)
        h = np.einsum("nk,kij->nij", w_all[lo:hi], lam)
        ev, vec = np.linalg.eigh(h)
        ph = np.exp(1j * eps * ev)
        u = np.einsum("nik,nk,njk->nij", vec, ph, np.conj(vec))
        out[lo:hi] = _reunitarise(u)

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(work, range(0, n, chunk)))
    return out.reshape(tuple(shape) + (3, 3))


def random_gauge(dims, eps, seed):
    """Synthetic gauge field of the given lattice, shape (V, 4, 3, 3)."""
    rng = np.random.default_rng(int(seed))
    return random_su3((lattice_volume(dims), 4), float(eps), rng)


def unit_gauge(dims):
    v = lattice_volume(dims)
    u = np.zeros((v, 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1
    return u


def random_gauge_transform(dims, seed, eps=2.0):
    """One SU(3) matrix per site, shape (V, 3, 3)."""
    rng = np.random.default_rng(int(seed) + 7919)
    return random_su3((lattice_volume(dims),), float(eps), rng)


def random_spinor(dims, seed, nrhs=None):
    """Complex Gaussian spinor field(s), shape (V, 4, 3) or (nrhs, V, 4, 3)."""
    rng = np.random.default_rng(int(seed) + 104729)
    v = lattice_volume(dims)
    shape = (v, 4, 3) if nrhs is None else (int(nrhs), v, 4, 3)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)
