"""Pins of the Schwarz alternating procedure and the flexible GCR of the
oracle (oracle/schwarz.py) against dense linear algebra:
  * one SAP cycle with exact block solves = the block Gauss-Seidel solve with
    [[A, 0], [C, E]] (black blocks first, Eq. domdec); two cycles = that step
    applied again to the residual;
  * GCR without preconditioner solves a dense system like numpy.linalg.solve,
    with a residual norm that never grows, with and without restarts;
  * SAP-preconditioned GCR solves D x = b like numpy.linalg.solve on 4^4, in
    far fewer iterations than plain GCR, also when the preconditioner changes
    from one iteration to the next (flexible).
"""
import numpy as np
import pytest

from oracle import dirac, geometry, schwarz
from paper_1112_1243_gb300 import synthetic

KAPPA = 0.12
CASES = [((4, 4, 4, 4), (2, 2, 2, 2), 0.4), ((8, 4, 4, 4), (4, 4, 4, 4), 0.4)]


def dd_vec(v, lat):
    return v[lat.dd_order].reshape(-1)


@pytest.mark.parametrize("dims,block,eps", CASES)
def test_sap_cycles_are_block_gauss_seidel(dims, block, eps):
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, eps, 41)
    rho = synthetic.random_spinor(dims, 42)
    D = dirac.dense_D(U, lat, KAPPA)
    A, B, C, E = dirac.dd_blocks(D, lat)
    nb = A.shape[0]
    L = np.zeros_like(D)
    L[:nb, :nb], L[nb:, :nb], L[nb:, nb:] = A, C, E
    idx = dirac.component_index(lat.dd_order)
    Dp = D[np.ix_(idx, idx)]
    blocks = schwarz.BlockSolver(U, lat, KAPPA)
    z1 = schwarz.sap(U, lat, KAPPA, rho, 1, blocks)
    ref1 = np.linalg.solve(L, dd_vec(rho, lat))
    assert np.max(np.abs(dd_vec(z1, lat) - ref1)) < 1e-12 * np.max(np.abs(ref1))
    z2 = schwarz.sap(U, lat, KAPPA, rho, 2, blocks)
    ref2 = ref1 + np.linalg.solve(L, dd_vec(rho, lat) - Dp @ ref1)
    assert np.max(np.abs(dd_vec(z2, lat) - ref2)) < 1e-12 * np.max(np.abs(ref2))
    # the cycles converge to D^{-1} rho (block Gauss-Seidel converges here)
    z8 = schwarz.sap(U, lat, KAPPA, rho, 8, blocks)
    exact = np.linalg.solve(Dp, dd_vec(rho, lat))
    e2 = np.linalg.norm(dd_vec(z2, lat) - exact)
    assert np.linalg.norm(dd_vec(z8, lat) - exact) < 1e-3 * e2


def test_gcr_matches_dense_solve_and_never_grows():
    rs = np.random.default_rng(5)
    n = 80
    A = np.eye(n) * 3 + (rs.standard_normal((n, n)) + 1j * rs.standard_normal((n, n))) / np.sqrt(n)
    b = rs.standard_normal(n) + 1j * rs.standard_normal(n)
    ref = np.linalg.solve(A, b)
    for nkv in (100, 6):
        hist = []
        x, it, res = schwarz.fgcr(lambda v: A @ v, lambda r: r, b, tol=1e-13, nkv=nkv, maxit=400, history=hist)
        assert res <= 1e-13 and np.max(np.abs(x - ref)) < 1e-11 * np.max(np.abs(ref))
        assert all(h2 <= h1 * (1 + 1e-12) for h1, h2 in zip(hist, hist[1:]))
    # without restarts GCR is exact after n directions (Krylov space of dimension n)
    x, it, res = schwarz.fgcr(lambda v: A @ v, lambda r: r, b, tol=1e-30, nkv=n, maxit=n)
    assert it == n and np.max(np.abs(x - ref)) < 1e-9 * np.max(np.abs(ref))


@pytest.mark.slow
def test_sap_gcr_solves_wilson_system():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.4, 43)
    b = synthetic.random_spinor(dims, 44)
    kappa = 0.13
    D = dirac.dense_D(U, lat, kappa)
    ref = np.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    x, it, res = schwarz.sap_gcr_solve(U, lat, kappa, b, tol=1e-12, ncy=2, nkv=8)
    assert res <= 1e-12
    assert np.max(np.abs(x - ref)) < 1e-10 * np.max(np.abs(ref))
    A = lambda v: dirac.apply_D(U, v, lat, kappa)
    _, it_plain, res_plain = schwarz.fgcr(A, lambda r: r, b, tol=1e-12, nkv=8, maxit=2000)
    assert res_plain <= 1e-12 and it < it_plain / 3, (it, it_plain)
    # flexible: a preconditioner with 1, 2, 3, 1, 2, 3, ... cycles
    blocks = schwarz.BlockSolver(U, lat, kappa)
    calls = {"k": 0}

    def varying(r):
        calls["k"] += 1
        return schwarz.sap(U, lat, kappa, r, 1 + calls["k"] % 3, blocks)

    x2, it2, res2 = schwarz.fgcr(A, varying, b, tol=1e-12, nkv=8)
    assert res2 <= 1e-12 and np.max(np.abs(x2 - ref)) < 1e-10 * np.max(np.abs(ref))
