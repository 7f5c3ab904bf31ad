"""Oracle pins for the Wilson-Dirac operator and its decompositions.

Pins: the free-field (U = 1) momentum-space form and spectrum, gamma5-
hermiticity, gauge covariance and gauge invariance of det D, the even-odd
identity det D = det Dtilde, and the Schur factorisation of Eq. ddfactor
checked with LAPACK determinants (numpy slogdet) of independently built
dense matrices.
"""
import itertools

import numpy as np
import pytest

from oracle import dirac, geometry
from oracle.gamma import GAMMA_AXIS, GAMMA5
from oracle.solvers import cgnr
from paper_1112_1243_gb300 import synthetic

KAPPA = 0.12


def _momenta(dims, bc_time=-1):
    ps = []
    for n in itertools.product(*[range(L) for L in dims]):
        p = [2 * np.pi * n[a] / dims[a] for a in range(3)]
        p.append((2 * n[3] + (1 if bc_time == -1 else 0)) * np.pi / dims[3])
        ps.append(np.array(p))
    return ps


def test_free_field_plane_waves():
    """D e^{ipx} u = e^{ipx} [1 - 2k sum cos p + 2ik sum gamma sin p] u."""
    dims = (4, 2, 6, 4)
    lat = geometry.Lattice(dims, (2, 2, 6, 2))
    U = synthetic.unit_gauge(dims)
    rs = np.random.default_rng(0)
    for p in _momenta(dims)[::7]:
        u = rs.standard_normal((4, 3)) + 1j * rs.standard_normal((4, 3))
        phase = np.exp(1j * lat.coords @ p)
        psi = phase[:, None, None] * u[None]
        out = dirac.apply_D(U, psi, lat, KAPPA)
        Dp = (1 - 2 * KAPPA * np.cos(p).sum()) * np.eye(4) + 2j * KAPPA * sum(GAMMA_AXIS[a] * np.sin(p[a]) for a in range(4))
        expect = phase[:, None, None] * (Dp @ u)[None]
        assert np.max(np.abs(out - expect)) < 1e-13


def test_free_field_determinant_closed_form():
    """ln|det D| = 6 sum_p ln(a^2 + 4k^2 sum sin^2 p), a = 1 - 2k sum cos p."""
    dims = (4, 4, 4, 4)
    lat = geometry.Lattice(dims, (2, 2, 2, 2))
    D = dirac.dense_D(synthetic.unit_gauge(dims), lat, KAPPA)
    ld = dirac.logabsdet(D)
    ref = 0.0
    for p in _momenta(dims):
        a = 1 - 2 * KAPPA * np.cos(p).sum()
        ref += 6 * np.log(a * a + 4 * KAPPA ** 2 * np.sum(np.sin(p) ** 2))
    assert abs(ld - ref) < 1e-9 * abs(ref)
    # the eigenvalues of D^dag D are a^2 + b^2, each 12-fold
    ev = np.sort(np.linalg.eigvalsh(D.conj().T @ D))
    refev = np.sort(np.repeat([(1 - 2 * KAPPA * np.cos(p).sum()) ** 2 + 4 * KAPPA ** 2 * np.sum(np.sin(p) ** 2)
                               for p in _momenta(dims)], 12))
    assert np.max(np.abs(ev - refev)) < 1e-12


@pytest.fixture(scope="module")
def small():
    dims = (4, 4, 4, 4)
    lat = geometry.Lattice(dims, (2, 2, 2, 2))
    U = synthetic.random_gauge(dims, 0.4, 1)
    D = dirac.dense_D(U, lat, KAPPA)
    return lat, U, D


def test_stencil_matches_dense(small):
    lat, U, D = small
    psi = synthetic.random_spinor(lat.dims, 3)
    out = dirac.apply_D(U, psi, lat, KAPPA)
    assert np.max(np.abs(out.reshape(-1) - D @ psi.reshape(-1))) < 1e-13
    outd = dirac.apply_Ddag(U, psi, lat, KAPPA)
    assert np.max(np.abs(outd.reshape(-1) - D.conj().T @ psi.reshape(-1))) < 1e-13


def test_gamma5_hermiticity(small):
    lat, U, D = small
    G5 = np.kron(np.eye(lat.V), np.kron(GAMMA5, np.eye(3)))
    assert np.max(np.abs(G5 @ D @ G5 - D.conj().T)) < 1e-14
    # hence det D is real
    sign, _ = np.linalg.slogdet(D)
    assert abs(sign.imag) < 1e-10


def test_gauge_covariance_and_invariance(small):
    lat, U, D = small
    g = synthetic.random_gauge_transform(lat.dims, 5)
    Ug = dirac.gauge_transform_links(U, g, lat)
    psi = synthetic.random_spinor(lat.dims, 4)
    lhs = dirac.apply_D(Ug, dirac.gauge_transform_spinor(psi, g), lat, KAPPA)
    rhs = dirac.gauge_transform_spinor(dirac.apply_D(U, psi, lat, KAPPA), g)
    assert np.max(np.abs(lhs - rhs)) < 1e-13
    ld = dirac.logabsdet(D)
    ldg = dirac.logabsdet(dirac.dense_D(Ug, lat, KAPPA))
    assert abs(ld - ldg) < 1e-10 * abs(ld)


def test_even_odd(small):
    lat, U, D = small
    H_eo, H_oe, Dt = dirac.dense_even_odd(D, lat, KAPPA)
    assert abs(dirac.logabsdet(D) - dirac.logabsdet(Dt)) < 1e-10
    # D^{-1} b through the even sites: x_e = Dt^{-1}(b_e + k H_eo b_o), x_o = b_o + k H_oe x_e
    b = synthetic.random_spinor(lat.dims, 6)
    ev = np.nonzero(lat.parity == 0)[0]
    od = np.nonzero(lat.parity == 1)[0]
    be = b[ev].reshape(-1)
    bo = b[od].reshape(-1)
    xe = np.linalg.solve(Dt, be + KAPPA * H_eo @ bo)
    xo = bo + KAPPA * H_oe @ xe
    x = np.empty_like(b)
    x[ev] = xe.reshape(-1, 4, 3)
    x[od] = xo.reshape(-1, 4, 3)
    assert np.max(np.abs(x.reshape(-1) - np.linalg.solve(D, b.reshape(-1)))) < 1e-12


def test_dirichlet_blocks(small):
    lat, U, D = small
    A, B, C, E = dirac.dd_blocks(D, lat)
    n = 12 * lat.block_sites
    nb = len(lat.black_blocks)
    for k, blk in enumerate(lat.black_blocks):
        Db = dirac.dense_dirichlet_block(U, lat, KAPPA, blk)
        assert np.max(np.abs(A[k * n:(k + 1) * n, k * n:(k + 1) * n] - Db)) < 1e-15
        assert np.max(np.abs(Db - dirac.dense_block_operator(D, lat, blk))) < 1e-15
        off = np.delete(A[k * n:(k + 1) * n], np.s_[k * n:(k + 1) * n], axis=1)
        assert np.all(off == 0)
    for k, blk in enumerate(lat.white_blocks):
        Db = dirac.dense_dirichlet_block(U, lat, KAPPA, blk)
        assert np.max(np.abs(E[k * n:(k + 1) * n, k * n:(k + 1) * n] - Db)) < 1e-15
    # the stencil split: intra + inter = all hops
    psi = synthetic.random_spinor(lat.dims, 8)
    full = dirac.apply_D(U, psi, lat, KAPPA)
    split = dirac.apply_D_dirichlet(U, psi, lat, KAPPA) + dirac.apply_D_inter(U, psi, lat, KAPPA)
    assert np.max(np.abs(full - split)) < 1e-14


@pytest.mark.parametrize("dims,block,eps", [((4, 4, 4, 4), (2, 2, 2, 2), 0.4),
                                            ((8, 4, 4, 4), (4, 4, 4, 4), 0.3)])
def test_schur_factorisation(dims, block, eps):
    """Eq. ddfactor: ln|det D| = sum_b ln|det D_b| + ln|det Dhat|."""
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, eps, 11)
    D = dirac.dense_D(U, lat, KAPPA)
    Dh = dirac.dense_schur(D, lat)
    lhs = dirac.logabsdet(D)
    rhs = sum(dirac.logabsdet(dirac.dense_dirichlet_block(U, lat, KAPPA, b)) for b in range(lat.nblocks))
    rhs += dirac.logabsdet(Dh)
    assert abs(lhs - rhs) < 1e-9 * abs(lhs) + 1e-9


def test_cgnr_solves_against_dense(small):
    lat, U, D = small
    b = synthetic.random_spinor(lat.dims, 9)
    A = lambda v: dirac.apply_D(U, v, lat, KAPPA)
    Ad = lambda v: dirac.apply_Ddag(U, v, lat, KAPPA)
    x, it, res = cgnr(A, Ad, b, tol=1e-13)
    assert res <= 1e-13
    ref = np.linalg.solve(D, b.reshape(-1))
    assert np.max(np.abs(x.reshape(-1) - ref)) < 1e-11
