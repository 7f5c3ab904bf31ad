"""Pins of the oracle's Markov-chain composition (Sec. 2, Sec. 3, Sec. 4,
Eq. 4step, Eq. ddrec, Eq. param) against the mathematics, not against the GPU.

* restore_rejected_blocks: the written-out definition (link by link), and the
  decoupling of the blocks: after the restore, the exact block log-ratio of a
  rejected block is exactly 0 and that of an accepted block is unchanged
  (the Dirichlet operator of a block holds only the links inside it).
* hierarchical_step / recursive_step, composition: with the proposal and the
  block decisions replaced by fixed stand-ins, the filters see (current,
  proposal), rejected blocks go back to the current links on exactly their
  active links, and the global step estimates (U0, U_final) in that order;
  mutants of the oracle with a swapped pair or a restore from the proposal
  fail these checks.
* Monte Carlo over the random streams (independent noise per seed):
  E[exp(sum_i ln r_i)] = det(Dhat'^dag Dhat') / det(Dhat^dag Dhat) (the
  estimator is unbiased, Sec. 4), E[min(1, exp(sum ln r))] <= min(1, exact)
  (Jensen: the stochastic acceptance is below the exact one, Sec. 4), and the
  sample mean and variance of sum_i ln r_i equal their closed forms
  -sum_i tr(M_i^dag M_i - 1) and sum_i ||M_i^dag M_i - 1||_F^2; the closed
  forms themselves show the O(1/N) bias and N Var = const of Eq. param.
  The same unbiasedness for the step-2 block-Schur estimates of the
  recursion (Eq. ddrec).
"""
import inspect
import math
import textwrap

import numpy as np
import pytest

import chain_support as cs
from oracle import accept, chain, dirac, estimator, geometry, heatbath, interp, recursive, rng
from paper_1112_1243_gb300 import synthetic

KAPPA = 0.12


def identity_field(U):
    return np.broadcast_to(np.eye(3, dtype=np.complex128), U.shape).copy()


def towards_identity(U, mask, t):
    """Links of `mask` moved a fraction t along the geodesic to the identity
    (a systematic change of the fermion determinant)."""
    out = np.array(U, copy=True)
    out[mask] = interp.interpolate(U, identity_field(U), t, mask)[mask]
    return out


# ---------------------------------------------------------------- restore
@pytest.mark.parametrize("dims,block", [((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 4, 4, 4), (4, 4, 4, 4))])
def test_restore_rejected_blocks_definition(dims, block):
    lat = geometry.Lattice(dims, block)
    U_old = synthetic.random_gauge(dims, 0.5, 11)
    U_new = synthetic.random_gauge(dims, 0.5, 12)     # differs on every link
    rs = np.random.default_rng(13)
    for _ in range(4):
        acc = rs.random(lat.nblocks) < 0.5
        got = accept.restore_rejected_blocks(U_new, U_old, lat, acc)
        assert np.array_equal(got, cs.restore_by_definition(U_new, U_old, lat, acc))
    assert np.array_equal(accept.restore_rejected_blocks(U_new, U_old, lat, np.ones(lat.nblocks, bool)), U_new)
    none = accept.restore_rejected_blocks(U_new, U_old, lat, np.zeros(lat.nblocks, bool))
    assert np.array_equal(none[lat.active], U_old[lat.active])
    assert np.array_equal(none[~lat.active], U_new[~lat.active])


@pytest.mark.parametrize("dims,block", [((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 4, 4, 4), (4, 4, 4, 4))])
def test_restore_decouples_block_ratios(dims, block):
    """Exact block log-ratios after the restore: 0 for rejected blocks,
    unchanged for accepted ones (bit for bit: the same links enter)."""
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.4, 21)
    Up = cs.kicked(U, lat, lat.active, 0.3, 22)
    full = estimator.block_ln_ratios_exact(U, Up, lat, KAPPA)
    assert np.all(full != 0.0)
    acc = np.arange(lat.nblocks) % 3 != 1
    after = estimator.block_ln_ratios_exact(U, accept.restore_rejected_blocks(Up, U, lat, acc), lat, KAPPA)
    assert np.array_equal(after, np.where(acc, full, 0.0))


# ---------------------------------------------------- chain composition
def chain_composition_violations(step_fn, dims, block, n_inner=2, n_global=3, seed=5, step=3):
    """Run `step_fn` (hierarchical_step or a mutant) with fixed proposals,
    forced block decisions and recording estimators; return the list of
    departures from the composition of Eq. 4step / Sec. 5."""
    lat = geometry.Lattice(dims, block)
    U0 = synthetic.random_gauge(dims, 0.4, 31)
    passes = chain.colour_passes(lat)
    ncall = n_inner * len(passes)
    targets = [cs.kicked(U0, lat, lat.active, 0.3, 40 + k) for k in range(ncall)]
    rs = np.random.default_rng(50)
    patterns = [rs.random(lat.nblocks) < 0.5 for _ in range(ncall)]
    out = []
    saved = (heatbath.gauge_update, accept.block_accept, estimator.block_ln_ratios, estimator.det_ratio_estimate)
    k_prop = {"k": 0}

    def proposal(U, lat_, beta, n_hb, n_or, seed_, ctr, colour_mask=3, active=None):
        p = cs.FixedProposal(targets[k_prop["k"]])
        k_prop["k"] += 1
        return p(U, lat_, beta, n_hb, n_or, seed_, ctr, colour_mask=colour_mask, active=active)

    filt = cs.Recorder(lambda n: np.zeros(lat.nblocks))
    glob = cs.Recorder(lambda n: np.linspace(-0.3, 0.2, n))
    try:
        heatbath.gauge_update = proposal
        accept.block_accept = cs.ForcedDecisions(patterns)
        estimator.block_ln_ratios = filt
        estimator.det_ratio_estimate = glob
        U_next, rec = step_fn(U0, lat, KAPPA, 5.3, n_inner, 2, n_global, seed, step)
    finally:
        heatbath.gauge_update, accept.block_accept, estimator.block_ln_ratios, estimator.det_ratio_estimate = saved
    # the composition written out
    Ucur = np.array(U0, copy=True)
    k = 0
    for it in range(n_inner):
        for p, cm in enumerate(passes):
            sel = cs.colour_sel(lat, cm)[:, None] & lat.active
            Up = np.array(Ucur, copy=True)
            Up[sel] = targets[k][sel]
            c = filt.calls[k] if k < len(filt.calls) else None
            if c is None or not (np.array_equal(c["U"], Ucur) and np.array_equal(c["Up"], Up)):
                out.append(f"filter {it}/{p} did not see (current, proposal)")
            if c is not None and c["ctr"] != chain.counter(step, it, p):
                out.append(f"filter {it}/{p} counter")
            acc = np.where(np.isin(lat.block_colour, [c_ for c_ in (0, 1) if cm >> c_ & 1]), patterns[k], True)
            Ucur = cs.restore_by_definition(Up, Ucur, lat, acc)
            k += 1
    if len(glob.calls) != 1:
        return out + ["global estimate not called once"]
    g = glob.calls[0]
    if not np.array_equal(g["U"], U0):
        out.append("global estimate: first field is not U0")
    if not np.array_equal(g["Up"], Ucur):
        out.append("global estimate: second field is not the filtered field")
    if g["n"] != n_global or g["ctr"] != chain.counter(step, n_inner, 0):
        out.append("global estimate: factors or counter")
    if not np.array_equal(rec["ln_global"], np.linspace(-0.3, 0.2, n_global)):
        out.append("record does not hold the estimate")
    u = rng.accept_uniform(np.zeros(1, dtype=np.uint64), rng.PURPOSE_GLOBAL_ACCEPT, seed, chain.counter(step, n_inner, 0))[0]
    ok = math.log(u) < float(np.sum(np.linspace(-0.3, 0.2, n_global)))
    if rec["accept"] != ok:
        out.append("global decision")
    if not np.array_equal(U_next, Ucur if ok else U0):
        out.append("returned field")
    return out


LATTICES = [((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 4, 4, 4), (4, 4, 4, 4))]


@pytest.mark.parametrize("dims,block", LATTICES)
def test_hierarchical_step_composition(dims, block):
    assert chain_composition_violations(chain.hierarchical_step, dims, block) == []
    # a second random-stream seed (another global uniform)
    assert chain_composition_violations(chain.hierarchical_step, dims, block, seed=6) == []


def mutant(fn, module, old, new):
    src = textwrap.dedent(inspect.getsource(fn))
    assert old in src, old
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<mutant of {fn.__name__}>", "exec"), ns)
    return ns[fn.__name__]


@pytest.mark.parametrize("old,new", [
    ("det_ratio_estimate(U0, Ucur", "det_ratio_estimate(Ucur, U0"),                         # swapped pair
    ("restore_rejected_blocks(Up, Ucur, lat, acc)", "restore_rejected_blocks(Up, Up, lat, acc)"),   # restore from Up
    ("restore_rejected_blocks(Up, Ucur, lat, acc)", "restore_rejected_blocks(Ucur, Up, lat, acc)"),  # arguments swapped
    ("block_ln_ratios(Ucur, Up,", "block_ln_ratios(Up, Ucur,"),                              # filter pair swapped
])
def test_hierarchical_step_mutants_are_caught(old, new):
    bad = mutant(chain.hierarchical_step, chain, old, new)
    assert chain_composition_violations(bad, *LATTICES[0]) != []


def recursive_composition_violations(step_fn, n_inner=2, seed=5, step=2):
    tl = recursive.TwoLevel((8, 4, 4, 4), (4, 4, 4, 4), (2, 2, 2, 2))
    lat1, lat2 = tl.lat1, tl.lat2
    U0 = synthetic.random_gauge(lat1.dims, 0.4, 61)
    targets = [cs.kicked(U0, lat2, tl.active, 0.3, 70 + k) for k in range(n_inner)]
    rs = np.random.default_rng(80)
    sub_pat = [rs.random(lat2.nblocks) < 0.5 for _ in range(n_inner)]
    blk_pat = [np.array([True, False]), np.array([False, True])][:n_inner]
    kp = {"k": 0}

    def proposal(U, lat_, beta, n_hb, n_or, seed_, ctr, colour_mask=3, active=None):
        p = cs.FixedProposal(targets[kp["k"]])
        kp["k"] += 1
        return p(U, lat_, beta, n_hb, n_or, seed_, ctr, colour_mask=colour_mask, active=active)

    sub = cs.Recorder(lambda n: np.zeros(lat2.nblocks))
    bs = cs.Recorder(lambda n: np.zeros(lat1.nblocks))
    glob = cs.Recorder(lambda n: np.full(n, -0.1))
    forced_b = cs.ForcedDecisions(blk_pat)
    saved = (heatbath.gauge_update, accept.block_accept, estimator.block_ln_ratios, estimator.det_ratio_estimate,
             recursive.block_schur_ln_ratios, recursive.block_schur_accept)
    try:
        heatbath.gauge_update = proposal
        accept.block_accept = cs.ForcedDecisions(sub_pat)
        estimator.block_ln_ratios = sub
        estimator.det_ratio_estimate = glob
        recursive.block_schur_ln_ratios = lambda U, Up, tl_, kappa, n, seed_, ctr, **kw: bs(U, Up, tl_, kappa, n, seed_, ctr, **kw)
        recursive.block_schur_accept = lambda ln, seed_, ctr, cm, bcol: forced_b(ln, seed_, ctr, cm, bcol)
        step_fn.__globals__.update(block_schur_ln_ratios=recursive.block_schur_ln_ratios,
                                   block_schur_accept=recursive.block_schur_accept)
        U_next, rec = step_fn(U0, tl, KAPPA, 5.3, n_inner, 2, 2, 3, seed, step)
    finally:
        (heatbath.gauge_update, accept.block_accept, estimator.block_ln_ratios, estimator.det_ratio_estimate,
         recursive.block_schur_ln_ratios, recursive.block_schur_accept) = saved
        step_fn.__globals__.update(block_schur_ln_ratios=saved[4], block_schur_accept=saved[5])
    out = []
    Ucur = np.array(U0, copy=True)
    for it in range(n_inner):
        Up = np.array(Ucur, copy=True)
        Up[tl.active] = targets[it][tl.active]
        c = sub.calls[it]
        if not (np.array_equal(c["U"], Ucur) and np.array_equal(c["Up"], Up)):
            out.append(f"step 1, iteration {it}: sub-block filter did not see (current, proposal)")
        Up = cs.restore_by_definition(Up, Ucur, lat2, sub_pat[it])
        c = bs.calls[it]
        if not (np.array_equal(c["U"], Ucur) and np.array_equal(c["Up"], Up)):
            out.append(f"step 2, iteration {it}: block-Schur filter did not see (current, sub-filtered proposal)")
        Ucur = cs.restore_by_definition(Up, Ucur, lat1, blk_pat[it])
    g = glob.calls[0]
    if not (np.array_equal(g["U"], U0) and np.array_equal(g["Up"], Ucur)):
        out.append("step 3: global estimate did not see (U0, filtered field)")
    if g["ctr"] != chain.counter(step, n_inner, 0):
        out.append("step 3: counter")
    ok = rec["accept"]
    if not np.array_equal(U_next, Ucur if ok else U0):
        out.append("returned field")
    return out


def test_recursive_step_composition():
    assert recursive_composition_violations(recursive.recursive_step) == []


@pytest.mark.parametrize("old,new", [
    ("det_ratio_estimate(U0, Ucur", "det_ratio_estimate(Ucur, U0"),
    ("block_schur_ln_ratios(Ucur, Up,", "block_schur_ln_ratios(Up, Ucur,"),
    ("restore_rejected_blocks(Up, Ucur, lat2, acc_s)", "restore_rejected_blocks(Up, Up, lat2, acc_s)"),
    ("restore_rejected_blocks(Up, Ucur, lat1, acc_b)", "restore_rejected_blocks(Up, Up, lat1, acc_b)"),
])
def test_recursive_step_mutants_are_caught(old, new):
    bad = mutant(recursive.recursive_step, recursive, old, new)
    assert recursive_composition_violations(bad) != []


# ------------------------------------------------------------- Monte Carlo
def dense_path(U0, Up, lat, K):
    """Dhat at the K + 1 points of the interpolation path (dense)."""
    return [dirac.dense_schur(dirac.dense_D(interp.interpolate(U0, Up, k / K, lat.active), lat, KAPPA), lat)
            for k in range(K + 1)]


def closed_forms(Ds, N):
    """Exact ln R, E[sum ln r_i] and Var[sum ln r_i] for N factors taken on
    the points Ds[0], Ds[K/N], ... (complex Gaussian noise, <|eta|^2> = 1:
    E eta^dag A eta = tr A, Var = tr A^2 for Hermitian A)."""
    K = len(Ds) - 1
    st = K // N
    ld = [dirac.logabsdet(Ds[k]) for k in (0, K)]
    mean = var = 0.0
    for i in range(N):
        M = np.linalg.solve(Ds[(i + 1) * st], Ds[i * st])
        A = M.conj().T @ M - np.eye(M.shape[0])
        mean -= np.trace(A).real
        var += np.linalg.norm(A) ** 2
    return 2.0 * (ld[1] - ld[0]), mean, var


@pytest.fixture(scope="module")
def global_setup():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    lat = geometry.Lattice(dims, block)
    U = synthetic.random_gauge(dims, 0.4, 1)
    # the proposal moves the active links away from the identity: the
    # determinant ratio is below one
    U0 = towards_identity(U, lat.active, 0.1)
    target = U
    Ds = dense_path(U0, target, lat, 8)
    return lat, U0, target, Ds


@pytest.mark.slow
def test_interpolation_bias_and_variance_scale_as_one_over_N(global_setup):
    """Eq. param: the product of N factors is exact as N -> infinity, the
    bias of sum ln r_i and its variance fall like 1/N."""
    lat, U0, target, Ds = global_setup
    rows = [closed_forms(Ds, N) for N in (1, 2, 4, 8)]
    lnR = rows[0][0]
    assert all(abs(r[0] - lnR) < 1e-10 for r in rows)       # one exact ratio (telescoping)
    bias = [lnR - r[1] for r in rows]
    var = [r[2] for r in rows]
    for N, b, v in zip((1, 2, 4, 8), bias, var):
        assert b > 0                                            # E ln r < ln R (x - 1 >= ln x)
        assert abs(N * b / bias[-1] / 8 - 1) < 0.05 * (8 // N), (N, b)
        assert abs(N * v / (8 * var[-1]) - 1) < 0.05 * (8 // N), (N, v)
    assert bias[0] > 1.9 * bias[1] > 3.7 * bias[2]


@pytest.mark.slow
def test_global_step_unbiased_and_below_exact_acceptance(global_setup):
    """Monte Carlo over the random streams of the oracle's hierarchical step
    (fixed proposal, all blocks accepted, 2 factors): mean of exp(sum ln r)
    = exact ratio; mean of min(1, .) <= min(1, exact ratio); sample mean and
    variance of sum ln r = the closed forms.  A swapped pair would estimate
    the inverse ratio, many standard errors away."""
    lat, U0, target, Ds = global_setup
    N, nsamp = 2, 96
    lnR, mean_cf, var_cf = closed_forms(Ds, N)
    R = math.exp(lnR)
    assert R < 1.0
    samples = cs.run_pool(cs.global_sample, [(U0, lat, target, KAPPA, N, 1000 + s, 1e-10) for s in range(nsamp)])
    tot = np.array([np.sum(x) for x in samples])
    est = np.exp(tot)
    se = est.std(ddof=1) / math.sqrt(nsamp)
    assert abs(est.mean() - R) < 4 * se, (est.mean(), R, se)
    assert abs(est.mean() - 1.0 / R) > 10 * se            # the test tells the pair from its swap
    m = np.minimum(1.0, est)
    assert m.mean() <= min(1.0, R) + 3 * m.std(ddof=1) / math.sqrt(nsamp)
    assert abs(tot.mean() - mean_cf) < 4 * math.sqrt(var_cf / nsamp), (tot.mean(), mean_cf)
    # sample variance against the closed form (chi^2-like spread; 4 sigma)
    assert abs(tot.var(ddof=1) / var_cf - 1) < 4 * math.sqrt(2.0 / (nsamp - 1)) * 1.5


@pytest.mark.slow
def test_block_schur_step_unbiased():
    """Eq. ddrec, step 2 of Eq. 4step: for every block, the mean over the
    random streams of exp(ln r_b) from the oracle's recursive step equals the
    exact block-Schur ratio det(Dhat_b'^dag Dhat_b') / det(Dhat_b^dag Dhat_b)."""
    tl = recursive.TwoLevel((8, 4, 4, 4), (4, 4, 4, 4), (2, 2, 2, 2))
    U = synthetic.random_gauge(tl.lat1.dims, 0.4, 3)
    U0 = towards_identity(U, tl.active, 0.1)
    exact = recursive.block_schur_ln_ratios_exact(U0, U, tl, KAPPA)
    assert np.all(exact < 0)
    nsamp = 64
    samples = np.array(cs.run_pool(cs.block_schur_sample, [(U0, tl, U, KAPPA, 1, 2000 + s, 1e-10)
                                                          for s in range(nsamp)]))
    est = np.exp(samples)
    for b in range(tl.lat1.nblocks):
        se = est[:, b].std(ddof=1) / math.sqrt(nsamp)
        R = math.exp(exact[b])
        assert abs(est[:, b].mean() - R) < 4 * se, (b, est[:, b].mean(), R, se)
        assert abs(est[:, b].mean() - 1.0 / R) > 8 * se
