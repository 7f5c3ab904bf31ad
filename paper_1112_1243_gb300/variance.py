"""Variance of the stochastic global acceptance step against the number N of
interpolation factors, its extrapolation in 1/N and the exact acceptance
rate (Sec. 4, the paragraph of Eq. param; Sec. 5, the paragraph on the exact acceptance rate;
Eq. acceptance).

With N factors the variance of ln r = sum_i ln r_i over proposals and noise
behaves as sigma^2(N) = sigma_2^2 + c / N: the noise part falls like 1/N,
and sigma_2^2 is the exact variance of ln det(M^dag M) due to the gauge
fluctuations.  Via the Gaussian model the exact acceptance rate is
erfc(sqrt(sigma_2^2 / 8)); over volumes sigma_2^2(V) is fitted by a line
through zero.  The GPU does the estimates (dd_det_ratio_estimate), the
proposals (dd_gauge_update) and the thermalisation of the pure-gauge field
(dd_gauge_update on a handle whose active set is every link); the fits are
plain least squares on the host.

Usage: python -m paper_1112_1243_gb300.variance --dims 8 8 8 8 --block 4 4 4 4
"""
import argparse
import json
import math

import numpy as np


def fit_inverse_n(Ns, variances):
    """Least-squares fit sigma^2(N) = a + b / N; returns (a, b)."""
    Ns = np.asarray(Ns, dtype=np.float64)
    v = np.asarray(variances, dtype=np.float64)
    A = np.stack([np.ones_like(Ns), 1.0 / Ns], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, v, rcond=None)
    return float(a), float(b)


def fit_through_zero(x, y):
    """Slope c of y = c x (least squares, intercept fixed at zero)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.dot(x, y) / np.dot(x, x))


def exact_acceptance(sigma2):
    """erfc(sqrt(sigma^2 / 8)) of the Gaussian model (Eq. acceptance)."""
    return math.erfc(math.sqrt(max(sigma2, 0.0) / 8.0))


def thermalise(api, dims, block, beta, sweeps, n_or, seed, U, device=None):
    """Heat-bath (+ n_or over-relaxation) sweeps over every link of U (in place)."""
    h = api.dd_init(dims, block, 0.125, active_mode=api.DD_ACTIVE_ALL, features=api.DD_FEAT_SOLVE, device=device)
    for k in range(sweeps):
        api.dd_gauge_update(h, U, 3, beta, 1, n_or, seed, (1 << 40) + k)
    plaq = api.dd_plaquette(h, U)
    return float(plaq.item())


def sample_ln_ratios(api, h, U, beta, N, samples, seed, offset=0, n_block=4):
    """Sum over N factors of ln r_i of the global step for `samples`
    proposals: one heat-bath sweep on the active links of U followed by the
    block filter (n_block factors; rejected blocks restored), as the global
    step sees them (Sec. 5), or the raw proposal for n_block = 0; a fresh
    proposal and fresh noise per sample.  U is not changed."""
    out = []
    for s in range(samples):
        ctr = ((offset + s) << 20) | N
        Up = U.clone()
        api.dd_gauge_update(h, Up, 3, beta, 1, 0, seed, ctr)
        if n_block > 0:
            api.dd_block_filter(h, U, Up, 3, api.DD_FILTER_STOCHASTIC, n_block, seed, ctr)
        ln = api.dd_det_ratio_estimate(h, U, Up, N, seed, ctr, api.DD_EST_FACTORS)
        out.append(float(ln.sum().item()))
    return np.array(out)


def variance_scan(api, h, U, beta, Ns, samples, seed, n_block=4):
    """sigma^2(N) of the global step for every N, the 1/N extrapolation and
    the acceptance rates (estimated and exact)."""
    rows = []
    for N in Ns:
        x = sample_ln_ratios(api, h, U, beta, N, samples, seed, offset=1000 * N, n_block=n_block)
        rows.append({"N": int(N), "var": float(np.var(x, ddof=1)), "mean": float(np.mean(x)),
                     "acceptance_mc": float(np.mean(np.minimum(1.0, np.exp(x))))})
    a, b = fit_inverse_n([r["N"] for r in rows], [r["var"] for r in rows])
    return {"rows": rows, "sigma2_exact": a, "noise_coefficient": b, "acceptance_exact": exact_acceptance(a)}


def main():
    import torch

    from . import api, synthetic
    p = argparse.ArgumentParser()
    p.add_argument("--dims", type=int, nargs=4, default=[8, 8, 8, 8])
    p.add_argument("--block", type=int, nargs=4, default=[4, 4, 4, 4])
    p.add_argument("--beta", type=float, default=5.8)
    p.add_argument("--kappa", type=float, default=0.15462)
    p.add_argument("--therm", type=int, default=200)
    p.add_argument("--Ns", type=int, nargs="+", default=[1, 2, 4, 8])
    p.add_argument("--samples", type=int, default=16)
    p.add_argument("--seed", type=int, default=11)
    p.add_argument("--n-block", type=int, default=4, help="block-filter factors (0: unfiltered proposals)")
    args = p.parse_args()
    dev = torch.device("cuda", 0)
    U = torch.from_numpy(synthetic.unit_gauge(args.dims)).to(dev)
    plaq = thermalise(api, args.dims, args.block, args.beta, args.therm, 2, args.seed, U, device=dev)
    h = api.dd_init(args.dims, args.block, args.kappa, max_rhs=max(max(args.Ns), 4), inner_prec=api.DD_PREC_F16,
                    krylov=api.DD_KRYLOV_BICGSTAB, maxit=100000, device=dev)
    res = variance_scan(api, h, U, args.beta, args.Ns, args.samples, args.seed, n_block=args.n_block)
    res.update(dims=args.dims, block=args.block, beta=args.beta, kappa=args.kappa, plaquette=plaq,
               thermalisation_sweeps=args.therm, samples=args.samples, n_block=args.n_block)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
