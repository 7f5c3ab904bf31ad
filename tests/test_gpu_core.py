"""GPU parity of the geometry tables, the Wilson-Dirac operator in its
forms, the global solver, the noise stream, the link interpolation and the
plaquette, all through the C ABI, against the FP64 oracle.

Tolerances (relative 2-norms unless stated):
  * maps: bit-exact;
  * FP64 operator: 1e-12 (the FP64 kernels reorder sums, rounding ~1e-16 per term);
  * FP32 storage: 1e-6 (FP32 rounding of links and spinors, 2^-24 ~ 6e-8 per
    element, amplified by the 8-term sums);
  * FP16 storage: 2e-3 (11-bit mantissa, 2^-11 ~ 5e-4 per element);
  * solves: the oracle's own D gives ||b - D x|| / ||b|| <= tol_global = 1e-10;
  * noise: 1e-14 absolute (the Philox words are identical; libm's log/cos/sin
    on the two sides may differ by an ulp).
"""
import numpy as np
import pytest

from oracle import dirac, geometry, heatbath, interp, rng
from paper_1112_1243_gb300 import synthetic
from tests.gpu_util import dev, host, lib_api, rel_err

pytestmark = pytest.mark.gpu

CASES = [
    # dims, block, eps, kappa   (the first has a ragged last thread block)
    ((6, 4, 4, 10), (3, 2, 2, 5), 0.4, 0.12),
    ((4, 4, 4, 4), (2, 2, 2, 2), 0.4, 0.12),
    ((8, 8, 8, 8), (4, 4, 4, 4), 0.3, 0.13),
]


@pytest.fixture(scope="module")
def api():
    return lib_api()


@pytest.mark.parametrize("dims,block,eps,kappa", CASES)
def test_maps_bit_exact(api, dims, block, eps, kappa):
    h = api.dd_init(dims, block, kappa)
    m = api.dd_get_maps(h)
    lat = geometry.Lattice(dims, block)
    assert np.array_equal(m["nbr"][:, :, 0], lat.fwd)
    assert np.array_equal(m["nbr"][:, :, 1], lat.bwd)
    assert np.array_equal(m["sign"][:, :, 0], lat.sign_fwd.astype(np.int32))
    assert np.array_equal(m["sign"][:, :, 1], lat.sign_bwd.astype(np.int32))
    assert np.array_equal(m["dd_order"], lat.dd_order)
    assert np.array_equal(m["block_of"], lat.block_id)
    assert np.array_equal(m["active"], lat.active)


def test_active_modes_bit_exact(api):
    for dims, block, mode, omode in [((16, 16, 8, 8), (8, 8, 4, 4), api.DD_ACTIVE_PAPER, "paper"),
                                     ((16, 16, 16, 16), (8, 8, 8, 8), api.DD_ACTIVE_INNER6, "inner6"),
                                     ((8, 8, 8, 8), (4, 4, 4, 4), api.DD_ACTIVE_INTRA, "intra")]:
        h = api.dd_init(dims, block, 0.13, active_mode=mode)
        lat = geometry.Lattice(dims, block, active_mode=omode)
        assert np.array_equal(api.dd_get_maps(h)["active"], lat.active)


@pytest.mark.parametrize("dims,block,eps,kappa", CASES)
def test_dslash_all_forms(api, dims, block, eps, kappa):
    nrhs = 2
    h = api.dd_init(dims, block, kappa, max_rhs=nrhs)
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, eps, 2)
    psi = synthetic.random_spinor(dims, 5, nrhs=nrhs)
    Ud = dev(U)
    ev = np.nonzero(lat.parity == 0)[0]
    od = np.nonzero(lat.parity == 1)[0]
    ref_D = np.stack([dirac.apply_D(U, p, lat, kappa) for p in psi])
    ref_Dd = np.stack([dirac.apply_Ddag(U, p, lat, kappa) for p in psi])
    ref_int = np.stack([dirac.apply_D_inter(U, p, lat, kappa) for p in psi])
    # Dtilde on even sites, built from the oracle stencil with parity masks
    def dtilde(p, dag=False):
        full = np.zeros((lat.V, 4, 3), dtype=np.complex128)
        full[ev] = p
        if dag:
            full = dirac.apply_gamma5(full)
        t = dirac.hop(U, full, lat)
        t[ev] = 0
        t2 = dirac.hop(U, t, lat)
        out = full - kappa * kappa * t2
        if dag:
            out = dirac.apply_gamma5(out)
        return out[ev]
    pe = psi[:, ev]
    ref_Dt = np.stack([dtilde(p) for p in pe])
    ref_Dtd = np.stack([dtilde(p, True) for p in pe])
    tol = {api.DD_PREC_F64: 1e-12, api.DD_PREC_F32: 1e-6, api.DD_PREC_F16: 2e-3}
    for prec in (api.DD_PREC_F64, api.DD_PREC_F32, api.DD_PREC_F16):
        out = dev(np.zeros_like(psi))
        api.dd_apply_D(h, out, dev(psi), Ud, api.DD_OP_D, prec, nrhs)
        assert rel_err(host(out), ref_D) < tol[prec]
        api.dd_apply_D(h, out, dev(psi), Ud, api.DD_OP_DDAG, prec, nrhs)
        assert rel_err(host(out), ref_Dd) < tol[prec]
        api.dd_apply_D(h, out, dev(psi), Ud, api.DD_OP_INTER, prec, nrhs)
        assert rel_err(host(out), ref_int) < tol[prec]
        oute = dev(np.zeros_like(pe))
        api.dd_apply_D(h, oute, dev(pe), Ud, api.DD_OP_DTILDE, prec, nrhs)
        assert rel_err(host(oute), ref_Dt) < tol[prec]
        api.dd_apply_D(h, oute, dev(pe), Ud, api.DD_OP_DTILDE_DAG, prec, nrhs)
        assert rel_err(host(oute), ref_Dtd) < tol[prec]
    # Dirichlet block operators, per colour
    for cm in (1, 2, 3):
        out = dev(np.zeros_like(psi))
        api.dd_apply_D_block(h, out, dev(psi), Ud, cm, api.DD_PREC_F64, nrhs)
        ref = np.stack([dirac.apply_D_dirichlet(U, p, lat, kappa) for p in psi])
        sel = np.isin(lat.colour, [c for c in (0, 1) if cm >> c & 1])
        ref[:, ~sel] = 0
        assert rel_err(host(out), ref) < 1e-12


def test_dslash_elementwise_fp64(api):
    """Element-by-element FP64 check (not only the norm) on a ragged lattice."""
    dims, block, kappa = (6, 4, 4, 10), (3, 2, 2, 5), 0.12
    h = api.dd_init(dims, block, kappa)
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.5, 9)
    psi = synthetic.random_spinor(dims, 10)
    out = dev(np.zeros_like(psi))
    api.dd_apply_D(h, out, dev(psi), dev(U), api.DD_OP_D, api.DD_PREC_F64, 1)
    ref = dirac.apply_D(U, psi, lat, kappa)
    assert np.max(np.abs(host(out) - ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec,krylov", [(0, 0), (1, 0), (2, 0), (1, 1), (2, 1)])
def test_solve_true_residual(api, prec, krylov):
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.13
    nrhs = 3
    h = api.dd_init(dims, block, kappa, max_rhs=nrhs, tol_global=1e-10, krylov=krylov)
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.3, 2)
    b = synthetic.random_spinor(dims, 11, nrhs=nrhs)
    x = dev(np.zeros_like(b))
    it, res, rc = api.dd_solve(h, x, dev(b), dev(U), nrhs, prec)
    xh = host(x)
    for r in range(nrhs):
        true = np.linalg.norm(b[r] - dirac.apply_D(U, xh[r], lat, kappa)) / np.linalg.norm(b[r])
        assert true <= 1e-10 * 1.01, (prec, r, true, res)
        assert abs(true - res[r]) <= 1e-11 + 0.1 * true
    assert it > 0


def test_noise_stream(api):
    dims = (6, 4, 4, 10)
    h = api.dd_init(dims, (3, 2, 2, 5), 0.12, max_rhs=2)
    V = int(np.prod(dims))
    eta = dev(np.zeros((2, V, 4, 3), dtype=np.complex128))
    api.dd_noise(h, eta, 2, rng.PURPOSE_USER_NOISE, 123456789012345, 77)
    got = host(eta)
    for r in range(2):
        ref = rng.spinor_noise(np.arange(V), rng.PURPOSE_USER_NOISE, r, 123456789012345, 77)
        assert np.max(np.abs(got[r] - ref)) < 1e-14


def test_interpolation(api):
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    h = api.dd_init(dims, block, 0.13)
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.3, 2)
    Up, _ = heatbath.gauge_update(U, lat, 5.3, 1, 0, 3, 1)
    Ut = dev(np.zeros_like(U))
    for i, n in [(0, 4), (1, 4), (3, 7), (5, 5), (1, 2)]:
        api.dd_interpolate(h, Ut, dev(U), dev(Up), i, n)
        ref = interp.interpolate(U, Up, i / n, lat.active)
        got = host(Ut)
        assert np.max(np.abs(got - ref)) < 1e-12, (i, n, np.max(np.abs(got - ref)))
        if i in (0, n):
            assert np.array_equal(got, ref)


def test_interpolation_far_apart(api):
    """Links far apart (phases near pi): compare with the oracle and check SU(3)."""
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    h = api.dd_init(dims, block, 0.12)
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 3.0, 4)
    Up = synthetic.random_gauge(dims, 3.0, 5)
    Ut = dev(np.zeros_like(U))
    api.dd_interpolate(h, Ut, dev(U), dev(Up), 2, 5)
    ref = interp.interpolate(U, Up, 0.4, lat.active)
    got = host(Ut)
    err = np.max(np.abs(got - ref), axis=(2, 3))
    assert np.max(err) < 1e-10
    a = got[lat.active]
    assert np.max(np.abs(np.linalg.det(a) - 1)) < 1e-12


def test_lean_workspace_features(api):
    """A handle planned for solves only has a smaller workspace, solves, and
    refuses the estimator with DD_ERR_UNSUPPORTED (no out-of-plan access)."""
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.13
    full = api.dd_init(dims, block, kappa, max_rhs=2)
    lean = api.dd_init(dims, block, kappa, max_rhs=2, features=api.DD_FEAT_SOLVE)
    assert lean.workspace.numel() < full.workspace.numel() / 2
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.3, 2)
    b = synthetic.random_spinor(dims, 11)
    x = dev(np.zeros_like(b))
    api.dd_solve(lean, x, dev(b), dev(U), 1, api.DD_PREC_F16)
    true = np.linalg.norm(b - dirac.apply_D(U, host(x), lat, kappa)) / np.linalg.norm(b)
    assert true <= 1.01e-10
    with pytest.raises(api.DDError) as e:
        api.dd_det_ratio_estimate(lean, dev(U), dev(U), 1, 1, 1)
    assert e.value.code == api.DD_ERR_UNSUPPORTED


def test_plaquette(api):
    dims = (6, 4, 4, 10)
    h = api.dd_init(dims, (3, 2, 2, 5), 0.12)
    lat = geometry.Lattice(dims, (3, 2, 2, 5))
    U = synthetic.random_gauge(dims, 0.6, 8)
    got = float(host(api.dd_plaquette(h, dev(U)))[0])
    assert abs(got - heatbath.plaquette_mean(U, lat)) < 1e-14
