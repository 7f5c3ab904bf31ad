"""Writes global_estimates.json: oracle values of the global stochastic
estimate (Sec. 4, Eq. param; the delta form of the Schur step) on two
workloads, for the GPU parity tests at sizes the oracle cannot finish inside
a test run.  Calls only the oracle (and the shared seeded input synthesis).

Per workload and factor i it stores
  ln_i        the oracle's ln r_i (estimator.ln_factor_delta, solves to 1e-14)
  eta_norm    |eta_i|
  s_norm      ||s_i||, s = B'E'^{-1}C' eta - A'A^{-1}BE^{-1}C eta (the source
              of the global solve)
  dinv_norm   ||D[U_{i+1}]^{-1}|| = 1 / sqrt(lambda_min(D^dag D)), lambda_min
              by Lanczos (scipy eigsh on the oracle's normal operator)
The proposal changes the active links only: U' = R U there, R = exp(i eps H)
from the seeded synthesis (numpy products only, identical on every host).

Usage:  python tests/golden/make_global_estimates.py [--workers 8]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CASES = {
    # 8^4 lattice, 4^4 blocks (active set of Sec. 3), kappa 0.13
    "8x4": dict(dims=(8, 8, 8, 8), block=(4, 4, 4, 4), kappa=0.13, eps=0.3, seed=2, kick_eps=0.15, kick_seed=21,
                n=2, noise_seed=9, ctr=4),
    # 16^4 lattice, 8^4 blocks (6^4 active sub-blocks), kappa 0.135, eps 0.25 (mixed-vs-FP64 workload)
    "16x8": dict(dims=(16, 16, 16, 16), block=(8, 8, 8, 8), kappa=0.135, eps=0.25, seed=3, kick_eps=0.15,
                 kick_seed=31, n=2, noise_seed=5, ctr=7),
}


def fields(case):
    import numpy as np
    from oracle import geometry
    from paper_1112_1243_gb300 import synthetic
    lat = geometry.Lattice(case["dims"], case["block"])
    U = synthetic.random_gauge(case["dims"], case["eps"], case["seed"])
    R = synthetic.random_gauge(case["dims"], case["kick_eps"], case["kick_seed"])
    Up = np.array(U, copy=True)
    Up[lat.active] = R[lat.active] @ U[lat.active]
    return lat, U, Up


def factor_fields(case, i):
    from oracle.interp import interpolate
    lat, U, Up = fields(case)
    n = case["n"]
    return lat, interpolate(U, Up, i / n, lat.active), interpolate(U, Up, (i + 1) / n, lat.active)


def task(arg):
    name, i, what = arg
    import numpy as np
    from oracle import dirac, estimator
    case = CASES[name]
    lat, Ui, Uj = factor_fields(case, i)
    t0 = time.time()
    if what == "ln":
        eta = estimator.global_noise(lat, i, case["noise_seed"], case["ctr"])
        ln = estimator.ln_factor_delta(Ui, Uj, eta, lat, case["kappa"], tol=1e-14)
        s = estimator.delta_source(Ui, Uj, eta, lat, case["kappa"], tol=1e-14)
        out = {"ln": float(ln), "eta_norm": float(np.linalg.norm(eta)), "s_norm": float(np.linalg.norm(s))}
    else:
        from scipy.sparse.linalg import LinearOperator, eigsh
        shape = (lat.V * 12, lat.V * 12)

        def normal(v):
            psi = v.reshape(lat.V, 4, 3)
            return dirac.apply_Ddag(Uj, dirac.apply_D(Uj, psi, lat, case["kappa"]), lat, case["kappa"]).reshape(-1)

        op = LinearOperator(shape, matvec=normal, dtype=np.complex128)
        v0 = np.ones(shape[0], dtype=np.complex128)
        lam = eigsh(op, k=1, which="SA", tol=1e-6, v0=v0, maxiter=20000, return_eigenvectors=False)[0]
        out = {"lambda_min": float(lam), "dinv_norm": float(1.0 / np.sqrt(lam))}
    out["seconds"] = time.time() - t0
    return name, i, what, out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=min(8, os.cpu_count() or 1))
    ap.add_argument("--cases", default=",".join(CASES))
    a = ap.parse_args()
    names = a.cases.split(",")
    jobs = [(n, i, w) for n in names for i in range(CASES[n]["n"]) for w in ("ln", "dinv")]
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    with mp.get_context("spawn").Pool(a.workers) as pool:
        res = pool.map(task, jobs, chunksize=1)
    path = os.path.join(HERE, "global_estimates.json")
    data = json.load(open(path)) if os.path.exists(path) else {}
    for n in names:
        case = dict(CASES[n])
        case["dims"], case["block"] = list(case["dims"]), list(case["block"])
        facs = [{} for _ in range(case["n"])]
        for name, i, what, out in res:
            if name == n:
                facs[i].update(out)
        data[n] = {"workload": case, "factors": facs,
                   "source": "oracle (tests/golden/make_global_estimates.py), solves to relative residual 1e-14"}
    with open(path, "w") as f:
        json.dump(data, f, indent=1)
    print(json.dumps(data, indent=1))


if __name__ == "__main__":
    main()
