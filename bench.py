#!/usr/bin/env python
"""Benchmark of the hierarchical domain-decomposed step on GB300.

Metric: global det-ratio estimates per second (one estimate = one
interpolation factor with its own noise vector, solved to true relative
residual 1e-10), mixed FP16/FP32 inner solver under FP64 defect correction.
A step is one full pass of the hot path: heat-bath proposal on the active
links, stochastic block filter (all Dirichlet block solves in one persistent
launch), the global Schur-complement estimate with n_global factors and the
global acceptance.  Default workload: 32^3 x 64 lattice, 8^4 blocks (6^4
active sub-blocks), eps = 0.2, kappa = 0.1355, 12 global factors, 4 block
factors, beta = 5.3.

Output: one JSON line (rank 0).  `--impl reference` times the FP64 numpy
oracle on a bounded sample of the same workload on the host cores.
Multi-GPU (torchrun): every rank runs its own independent chain (no data-path
collective); value = all ranks' estimates / max rank time (weak scaling).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "det-ratio estimates/s (global Schur step, residual 1e-10, mixed FP16/FP32 + FP64 defect correction)"

CONFIGS = {
    # name: lattice, blocks, eps, kappa, gauge seed, global factors, block factors
    "c2": dict(dims=(8, 8, 8, 8), block=(4, 4, 4, 4), eps=0.3, kappa=0.13, seed=2, n_global=16, n_block=4),
    "c3": dict(dims=(16, 16, 16, 16), block=(8, 8, 8, 8), eps=0.25, kappa=0.135, seed=3, n_global=8, n_block=4),
    "c5": dict(dims=(32, 32, 32, 64), block=(8, 8, 8, 8), eps=0.2, kappa=0.1355, seed=5, n_global=12, n_block=4),
    # smaller volume of the same physics for kernel captures (inputs still larger than L2)
    "c5s": dict(dims=(32, 32, 32, 48), block=(8, 8, 8, 8), eps=0.2, kappa=0.1355, seed=5, n_global=12, n_block=4),
}
BETA = 5.3
# algorithmic bytes per output site of the eo hop kernels (input spinor + 8
# links with two stored rows + output; FP16 spinor = 48 B + 4 B scale,
# FP16 link rows = 24 B, FP32 spinor = 96 B, FP64 spinor 192 B, FP64 link 144 B)
# algorithmic bytes per output site: input spinor once, 8 links, xpay input, output
# (kind 3, the double-float residual hop: the t = H_oe x form, FP64-sized vectors and links)
HOP_BYTES = {0: 52 + 8 * 24 + 52, 1: 52 + 8 * 24 + 96 + 96, 2: 192 + 8 * 144 + 192, 3: 192 + 8 * 144 + 192}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--config", default="c5", choices=sorted(CONFIGS))
    p.add_argument("--prec", default="f16", choices=["f16", "f32", "f64"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay measurement")
    p.add_argument("--no-tune", action="store_true", help="keep the default launch shapes")
    p.add_argument("--no-recursive", action="store_true", help="skip the step with one level of recursion")
    p.add_argument("--outer", default="f64", choices=["f64", "df64"],
                   help="arithmetic of the defect-correction residual of the timed step")
    p.add_argument("--no-outer-df64", action="store_true",
                   help="skip the extra measurement of the step with the double-float residual")
    p.add_argument("--tol-inner", type=float, default=1e-3,
                   help="residual reduction of one inner (FP32/FP16) solve inside the FP64 defect correction")
    p.add_argument("--fp64-steps", type=int, default=0,
                   help="also time this many steps with the plain FP64 solver (same workload)")
    p.add_argument("--no-batched-filter", action="store_true",
                   help="skip the uneven-block batched filter measurement")
    p.add_argument("--compare-config", default="c2,c3",
                   help="workloads of the mixed-versus-FP64 comparison, comma-separated ('' to skip)")
    p.add_argument("--krylov", default="bicgstab", choices=["cgnr", "bicgstab", "sap"],
                   help="inner Krylov method of the mixed-precision solves")
    p.add_argument("--no-lu", action="store_true", help="skip the timing of the dense LU check path (c1)")
    p.add_argument("--no-tol-block", action="store_true",
                   help="skip the measurement of the step with Dirichlet solves to 1e-10 instead of 1e-12")
    p.add_argument("--no-f32-storage", action="store_true",
                   help="skip the measurement of the step with FP32-storage inner solvers (tol_inner 1e-6)")
    p.add_argument("--no-sap", action="store_true",
                   help="skip the measurement of the step with SAP-preconditioned GCR global solves")
    p.add_argument("--sap-ncy", type=int, default=4, help="Schwarz cycles per SAP-GCR preconditioner application")
    p.add_argument("--sap-nmr", type=int, default=4, help="BiCGStab iterations per approximate SAP block solve")
    p.add_argument("--sap-nkv", type=int, default=6, help="directions of the flexible GCR before a restart")
    p.add_argument("--mode", default="step", choices=["step", "solve", "lu"],
                   help="step: the hierarchical step (the benchmark); solve: one-rhs global solves on a lean "
                        "handle (kernel captures and Dslash GB/s)")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit())
        smax = max(float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].strip().lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(self.samples)}


# ------------------------------------------------------------------ oracle arm
def oracle_sample(cfg, seconds=20.0):
    """Time the FP64 numpy oracle's Wilson operator at the full volume for a
    bounded number of applications; returns seconds per application and the count."""
    import numpy as np
    from oracle import dirac, geometry
    from paper_1112_1243_gb300 import synthetic
    lat = geometry.Lattice(cfg["dims"], cfg["block"])
    U = synthetic.random_gauge(cfg["dims"], cfg["eps"], cfg["seed"])
    psi = synthetic.random_spinor(cfg["dims"], 1)
    n, t = 0, 0.0
    while t < seconds and n < 50:
        t0 = time.perf_counter()
        psi = dirac.apply_D(U, psi, lat, cfg["kappa"])
        psi /= np.linalg.norm(psi)
        t += time.perf_counter() - t0
        n += 1
    return t / n, n, t


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def _oracle_factor(a):
    """One factor of the oracle's global estimate (delta form), timed alone;
    returns (seconds, ln r_i).  Runs in a worker process."""
    cfg, U, Up, i, n, seed, ctr, tol = a
    from oracle import estimator, geometry
    from oracle.interp import interpolate
    lat = geometry.Lattice(cfg["dims"], cfg["block"])
    Ui = interpolate(U, Up, i / n, lat.active)
    Uj = interpolate(U, Up, (i + 1) / n, lat.active)
    eta = estimator.global_noise(lat, i, seed, ctr)
    t0 = time.perf_counter()
    ln = estimator.ln_factor_delta(Ui, Uj, eta, lat, cfg["kappa"], tol=tol)
    return time.perf_counter() - t0, float(ln)


def oracle_estimate_rate(cfg, tol=1e-10, seed=1, ctr=0):
    """The FP64 numpy oracle's global stochastic estimate on a whole workload
    (no projection): the proposal (one oracle heat-bath sweep on the active
    links) is made first; then factor 0 alone on one thread, and all
    n_global factors at once, one process per core (start method spawn).
    Returns estimates/s for both and what was run."""
    import multiprocessing as mp
    from oracle import geometry, heatbath
    from paper_1112_1243_gb300 import synthetic
    lat = geometry.Lattice(cfg["dims"], cfg["block"])
    U = synthetic.random_gauge(cfg["dims"], cfg["eps"], cfg["seed"])
    Up, _ = heatbath.gauge_update(U, lat, BETA, 1, 0, seed, ctr)
    n = cfg["n_global"]
    t1, _ = _oracle_factor((cfg, U, Up, 0, n, seed, ctr, tol))
    cores = max(1, min(n, os.cpu_count() or 1))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            pool.map(abs, range(cores))          # workers started and imported before timing
            w0 = time.perf_counter()
            res = pool.map(_oracle_factor, [(cfg, U, Up, i, n, seed, ctr, tol) for i in range(n)], chunksize=1)
            wall = time.perf_counter() - w0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {"one_thread": 1.0 / t1, "all_cores": n / wall, "cores": cores, "seconds_one_factor": t1,
            "seconds_all_factors": wall, "factors": n, "tol": tol}


def site_hops_per_estimate_default(cfg_name):
    """Whole-lattice Wilson applications per global estimate, measured on the
    GPU path (global, Dirichlet and block-solver work) and recorded in
    profiles/; used by the reference arm, which runs without a GPU
    measurement of its own."""
    path = os.path.join(ROOT, "profiles", "work_per_estimate.json")
    try:
        with open(path) as f:
            return float(json.load(f)[cfg_name]["D_applications_per_estimate"])
    except Exception:
        return None


def run_reference(args, cfg):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    napp = site_hops_per_estimate_default(args.config)
    per_app, n, t = oracle_sample(cfg, seconds=15.0)
    steps = []
    for _ in range(args.warmup + args.steps):
        pa, _, _ = oracle_sample(cfg, seconds=5.0)
        steps.append(pa)
    per_app = sum(steps[args.warmup:]) / max(1, args.steps)
    if napp is None:
        print(json.dumps({"impl": "reference", "unavailable": "no recorded GPU work-per-estimate for this config"}))
        return 0
    est_per_s = 1.0 / (napp * per_app)
    V = math.prod(cfg["dims"])
    line = {
        "metric": METRIC, "value": est_per_s, "unit": "estimates/s", "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # one step of the GPU arm (n_global estimates) at the sampled rate
        "ms_per_step": 1e3 * cfg["n_global"] / est_per_s, "sample_seconds_per_step": per_app,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": config_dict(args, cfg, 1),
        "cpu_baseline": {"value": est_per_s, "unit": "estimates/s", "cores": 1, "kind": "oracle",
                         "sample": f"numpy FP64 oracle apply_D at V={V}: {per_app:.3f} s per application "
                                   f"(steps of >=5 s), scaled by {napp:.0f} Wilson applications per estimate "
                                   f"(GPU-measured work of the step: global, Dirichlet and block-solver "
                                   f"applications); one core", "projected": True},
        "e2e": {"value": est_per_s, "unit": "estimates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# FP64 hop: 1320 flops per site for the stencil (165 per hop) + 48 for the xpay term
FP64_HOP_FLOPS = 1368
FLOPS_PER_HOP = 165
# one BiCGStab iteration of the persistent block solver, per block site (FP32):
# two Dirichlet applications (1368 flops each at most) + the vector updates and
# inner products (about 960 flops over the 12 complex components)
BLOCK_ITER_FLOPS = 2 * FP64_HOP_FLOPS + 960
# unit counts and clock (152 SMs, 2070 MHz): FP64 2 FMA per SM per cycle,
# FP32 128 FMA per SM per cycle -- the fallback when the live probe fails
DERIVED_PEAKS = {"fp64_fma": 152 * 2 * 2 * 2.07e9 / 1e12, "fp32_fma": 152 * 128 * 2 * 2.07e9 / 1e12}


def hops_kept(block):
    """Hops per site that stay inside a block (of 8), averaged over the block."""
    return sum(2.0 * (1.0 - 1.0 / b) for b in block)


def kernel_models(block):
    """Timed kernel kinds -> (name, bound, algorithmic bytes per unit, flops
    per unit, unit).  Units: output sites of one right-hand side (hops); block
    sites x inner iterations (persistent block solver)."""
    k = hops_kept(block)
    return {
        0: ("hop_eo_kernel FP16 -> FP16, whole lattice", "hbm", HOP_BYTES[0], 1320, "site"),
        1: ("hop_eo_kernel FP16 -> FP32 + xpay, whole lattice", "hbm", HOP_BYTES[1], 1368, "site"),
        2: ("hop_eo_kernel FP64 (defect-correction residual), whole lattice", "fp64", HOP_BYTES[2], 1368, "site"),
        3: ("hop_df_kernel double-float residual, whole lattice", "fp32", HOP_BYTES[3], 8600, "site"),
        4: ("hop_eo_kernel FP64 (defect-correction residual), Dirichlet blocks", "fp64",
            192 + 144 * k + 192, 48 + FLOPS_PER_HOP * k, "site"),
        5: ("hop_eo_kernel FP16 -> FP16, Dirichlet blocks, one colour's sites", "hbm", 52 + 24 * k + 52,
            FLOPS_PER_HOP * k, "site"),
        6: ("hop_eo_kernel FP16 -> FP32 + xpay, Dirichlet blocks, one colour's sites", "hbm", 52 + 24 * k + 96 + 96,
            48 + FLOPS_PER_HOP * k, "site"),
        7: ("block_solve_kernel (persistent, FP32 BiCGStab + FP64 refinement)", "fp32", None, BLOCK_ITER_FLOPS,
            "block site x inner iteration"),
        8: ("hop_eo_kernel FP16 -> FP16, Dirichlet blocks, every site", "hbm", 52 + 24 * k + 52, FLOPS_PER_HOP * k,
            "site"),
        9: ("hop_eo_kernel FP16 -> FP32 + xpay, Dirichlet blocks, every site", "hbm", 52 + 24 * k + 96 + 96,
            48 + FLOPS_PER_HOP * k, "site"),
    }


def peaks_alu(stream):
    """FP64/FP32 FMA peaks measured live by the library (derived from unit
    counts and the maximum clock if the probe fails), and where they came from."""
    from paper_1112_1243_gb300 import api
    try:
        return api.dd_alu_peaks(stream), "measured live (dd_alu_peaks: FMA chains, CUDA events)"
    except api.DDError:
        return dict(DERIVED_PEAKS), "derived: SM count x FMA units per cycle x 2070 MHz"


def roofline_entry(kind, model, ms, launches, units, step_ms, hbm_peak, alu, alu_src):
    """Roofline entry of one timed kernel kind (None when nothing was timed)."""
    name, bound, bpu, fpu, unit = model
    if not (ms and ms > 0 and units and units > 0):
        return None
    e = {"kind": kind, "kernel": name, "launches_timed": launches, "total_ms": ms,
         "share_of_step": ms / step_ms if step_ms else None, "avg_launch_us": 1e3 * ms / max(1, launches),
         "units": units, "unit": unit}
    if bound == "hbm":
        ach = units * bpu / 1e9 / (ms / 1e3)
        e.update(bound="hbm", achieved=ach, peak=hbm_peak, unit_rate="GB/s", frac=ach / hbm_peak,
                 bytes_per_unit=bpu)
    else:
        key = "fp64_fma" if bound == "fp64" else "fp32_fma"
        ach = units * fpu / 1e12 / (ms / 1e3)
        e.update(bound="alu", pipe=key, achieved=ach, peak=alu[key], unit_rate="TFLOP/s", frac=ach / alu[key],
                 flops_per_unit=fpu, peak_source=alu_src)
        if bpu:
            e["GB_per_s"] = units * bpu / 1e9 / (ms / 1e3)
    return e


def replica_seeds(cfg, rank):
    """Seeds of the independent chain of one rank (replicas: no data-path
    exchange between ranks): gauge-field seed and random-stream seed."""
    return cfg["seed"] + 1000 * rank, cfg["seed"] * 7919 + rank


def max_over_ranks(t_ms, world, device=None):
    """The slowest rank's time (every rank gets it): the whole job is done
    when the last replica is."""
    if world <= 1:
        return float(t_ms)
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(units_per_rank, world, t_max_ms):
    """Whole-job throughput: the units all ranks processed over the slowest time."""
    return units_per_rank * world / (t_max_ms / 1e3)


def config_dict(args, cfg, world):
    """The workload description shared by both arms of the benchmark."""
    return {"workload": f"{args.config}: {'x'.join(map(str, cfg['dims']))} lattice, "
                        f"{'x'.join(map(str, cfg['block']))} blocks (6^4 active sub-blocks), eps {cfg['eps']}, "
                        f"kappa {cfg['kappa']}, beta {BETA}, {cfg['n_global']} global + {cfg['n_block']} block "
                        f"factors, residual 1e-10",
            "krylov": args.krylov,
            "l2": "inputs larger than L2 (gauge field alone 1.2 GB)", "chains": world}


# --------------------------------------------------------------------- GPU arm
def run_gpu(args, cfg):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1112_1243_gb300 import api, build, synthetic
    from paper_1112_1243_gb300.chain import HierarchicalStep

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    prec = {"f16": api.DD_PREC_F16, "f32": api.DD_PREC_F32, "f64": api.DD_PREC_F64}[args.prec]
    V = math.prod(cfg["dims"])
    Vh = V // 2
    nmax = max(cfg["n_global"], cfg["n_block"])
    stream = torch.cuda.current_stream(dev)
    krylov = {"cgnr": api.DD_KRYLOV_CGNR, "bicgstab": api.DD_KRYLOV_BICGSTAB, "sap": api.DD_KRYLOV_SAP_GCR}[args.krylov]
    outer = {"f64": api.DD_PREC_F64, "df64": api.DD_PREC_DF64}[args.outer]
    h = api.dd_init(cfg["dims"], cfg["block"], cfg["kappa"], max_rhs=nmax, inner_prec=prec,
                    block_prec=api.DD_PREC_F32, tol_global=1e-10, tol_block=1e-12, tol_inner=args.tol_inner,
                    maxit=40000, stream=stream, device=dev, krylov=krylov, outer_prec=outer,
                    sap_ncy=args.sap_ncy, sap_nmr=args.sap_nmr, sap_nkv=args.sap_nkv)
    U_np = synthetic.random_gauge(cfg["dims"], cfg["eps"], replica_seeds(cfg, rank)[0])
    U = torch.from_numpy(U_np).to(dev)
    tune = None
    if not args.no_tune:
        # launch shapes of the hop kernels and of the persistent block solver,
        # timed on this lattice (the block solver on one proposal's filter)
        Up_t = U.clone()
        api.dd_gauge_update(h, Up_t, 3, BETA, 1, 0, 4242, 0)
        tune = api.dd_autotune(h, api.DD_TUNE_HOP | api.DD_TUNE_BLOCK, U, Up_t, reps=10)
        del Up_t
    chain = HierarchicalStep(h, BETA, n_inner=1, n_block=cfg["n_block"], n_global=cfg["n_global"],
                             seed=replica_seeds(cfg, rank)[1])
    # roofline denominators of the ALU-bound kernels, measured on this GPU
    alu, alu_src = peaks_alu(stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for k in range(args.warmup):
        chain.step(U, k)
    barrier()
    api.dd_kernel_timer(h, 1, 0, 1)
    l0 = api.dd_launch_count(h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    acc = []
    ref_ln = []
    with ClockSampler(local) as clocks:
        e0.record(stream)
        for k in range(args.steps):
            ln, a = chain.step(U, args.warmup + k)
            ref_ln.append(ln.clone())
        e1.record(stream)
        barrier()
    t_ms = e0.elapsed_time(e1)
    launches = api.dd_launch_count(h) - l0
    timing = {kind: api.dd_kernel_timer(h, 2, kind) for kind in range(api.DD_TIMER_KIND_COUNT)}
    stats = {name: api.dd_solver_stats(h, k) for k, name in ((0, "global"), (1, "dirichlet"), (2, "block_solver"))}
    api.dd_kernel_timer(h, 0, 0)
    t_max = max_over_ranks(t_ms, world, dev)
    est = cfg["n_global"] * args.steps * world
    value = job_rate(cfg["n_global"] * args.steps, world, t_max)
    peak, peak_src = peaks()
    models = kernel_models(cfg["block"])
    # persistent block solver: its unit is a block site x inner iteration
    units = {k: timing[k][2] for k in timing}
    units[7] = stats["block_solver"]["site_iterations"]
    entries = [roofline_entry(k, models[k], timing[k][0], timing[k][1], units[k], t_ms, peak, alu, alu_src)
               for k in sorted(models)]
    entries = [e for e in entries if e]
    # the roofline line: the timed kernel kind with the most time in the step
    dom = max(entries, key=lambda e: e["total_ms"])
    kind = dom["kind"]
    ms_k, cnt_k, sites_k = timing[kind]
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "hop_traffic.json")) as f:
            tr = json.load(f)
        src = open(os.path.join(ROOT, "paper_1112_1243_gb300", "csrc", "dslash.cuh"), "rb").read()
        import hashlib
        if tr.get("dslash_sha256") == hashlib.sha256(src).hexdigest() and str(kind) in tr.get("bytes_per_site", {}):
            traffic = tr["bytes_per_site"][str(kind)] * (sites_k / max(1, cnt_k))
    except Exception:
        traffic = None
    # Wilson applications per estimate: whole-lattice and Dirichlet hops (two
    # hops of Vh sites = one application of V sites) and the persistent block
    # solver (two Dirichlet applications per inner iteration)
    hop_sites = sum(timing[k][2] for k in (0, 1, 2, 3, 4, 5, 6, 8, 9))
    blk_apps = 2.0 * stats["block_solver"]["site_iterations"]
    D_apps_per_est = (hop_sites / (2.0 * Vh) + blk_apps / V) / max(1, cfg["n_global"] * args.steps)
    iterations = {}
    for name, st in stats.items():
        n = st["systems"] if "systems" in st else st["items"]
        calls = st["solves"] if "solves" in st else st["items"]
        iterations[name] = dict(st, inner_per_system=st["inner_iterations"] / n if n else None,
                                outer_cycles_per_solve=st["outer_cycles"] / calls if calls else None)
    if dom["bound"] == "hbm":
        roofline = {"bound": "hbm", "kernel": dom["kernel"], "achieved": dom["achieved"], "peak": peak,
                    "unit": "GB/s", "frac": dom["frac"], "traffic": traffic,
                    "bytes_per_site": dom["bytes_per_unit"], "launches_timed": cnt_k,
                    "avg_launch_us": dom["avg_launch_us"], "share_of_step": dom["share_of_step"],
                    "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        roofline = {"bound": "alu", "kernel": dom["kernel"], "achieved": dom["achieved"], "peak": dom["peak"],
                    "unit": "TFLOP/s", "frac": dom["frac"], "traffic": traffic,
                    "flops_per_site": dom["flops_per_unit"], "launches_timed": cnt_k,
                    "avg_launch_us": dom["avg_launch_us"], "share_of_step": dom["share_of_step"],
                    "peak_source": dom["peak_source"]}
    line = {
        "metric": METRIC, "value": value, "unit": "estimates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f16": "f16-storage/f32", "f32": "f32", "f64": "f64"}[args.prec] + "+" + args.outer,
        "data": "synthetic",
        "config": config_dict(args, cfg, world),
        "roofline": roofline,
        "rooflines": entries,
        "alu_peaks": dict(alu, source=alu_src),
        "iterations": iterations,
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "D_applications_per_estimate": D_apps_per_est,
        "dslash_GBps": {name: (timing[k][2] * HOP_BYTES[k] / 1e9 / (timing[k][0] / 1e3) if timing[k][0] > 0 else None)
                        for k, name in ((0, "fp16_to_fp16"), (1, "fp16_to_fp32_xpay"), (2, "fp64"),
                                        (3, "double_float"))},
        "block_accept_rate_last_step": float(chain.acc_b.float().mean().item()),
        "autotune": tune,
    }
    # end to end through the public API with host buffers
    if not args.no_e2e:
        U_host = torch.empty(U.shape, dtype=U.dtype).pin_memory()
        U_host.copy_(U.cpu())
        ln_host = torch.empty(cfg["n_global"], dtype=torch.float64).pin_memory()
        acc_host = torch.empty(1, dtype=torch.uint8).pin_memory()
        U_dev = torch.empty_like(U)
        # untimed warm-up of the end-to-end path (first use of the pinned buffers)
        for k in range(min(args.warmup, 2)):
            chain.step_host(U_host, U_dev, 900 + k, ln_host, acc_host)
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for k in range(args.steps):
            chain.step_host(U_host, U_dev, 1000 + k, ln_host, acc_host)
        f1.record(stream)
        barrier()
        te = max_over_ranks(f0.elapsed_time(f1), world, dev)
        # the host<->device copies of one step alone (same buffers, no step)
        U_back = torch.empty_like(U_host).pin_memory()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for k in range(args.steps):
            U_dev.copy_(U_host, non_blocking=True)
            U_back.copy_(U_dev, non_blocking=True)
        c1.record(stream)
        c1.synchronize()
        line["e2e"] = {"value": est / (te / 1e3), "unit": "estimates/s",
                       "h2d_bytes_per_step": U.numel() * 16,
                       "d2h_bytes_per_step": U.numel() * 16 + cfg["n_global"] * 8 + 1,
                       "ms_per_step": te / args.steps,
                       "copy_ms_per_step": c0.elapsed_time(c1) / args.steps}
        del U_back
    # the same step recorded once as a CUDA graph (solver loops as device-side
    # conditional nodes) and replayed with advancing random streams
    if not args.no_graph:
        g = chain.capture(U)
        for k in range(args.warmup):
            chain.step_graph(2000 + k)
        barrier()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for k in range(args.steps):
            chain.step_graph(3000 + k)
        q1.record(stream)
        barrier()
        tg = max_over_ranks(q0.elapsed_time(q1), world, dev)
        st_code = api.dd_status(h)[0]
        line["graph"] = {"value": est / (tg / 1e3), "unit": "estimates/s", "ms_per_step": tg / args.steps,
                         "top_level_nodes": api.dd_graph_nodes(g), "device_status": st_code}
        api.dd_graph_destroy(g)
        del g  # the graph object holds the handle: release it with the handle
    if args.fp64_steps > 0:
        h64 = api.dd_init(cfg["dims"], cfg["block"], cfg["kappa"], max_rhs=nmax, inner_prec=api.DD_PREC_F64,
                          block_prec=api.DD_PREC_F32, tol_global=1e-10, tol_block=1e-12, maxit=40000,
                          stream=stream, device=dev)
        c64 = HierarchicalStep(h64, BETA, n_inner=1, n_block=cfg["n_block"], n_global=cfg["n_global"],
                               seed=replica_seeds(cfg, rank)[1])
        U64 = torch.from_numpy(U_np).to(dev)
        c64.step(U64, 0)
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for k in range(args.fp64_steps):
            c64.step(U64, 1 + k)
        g1.record(stream)
        barrier()
        line["fp64_value"] = cfg["n_global"] * args.fp64_steps / (g0.elapsed_time(g1) / 1e3)
        del h64
    del chain
    del h
    torch.cuda.empty_cache()
    # supplementary measurements: one that fails is recorded in the line as
    # {"error": ...} and the run goes on (the numbers above stay valid)
    if not args.no_outer_df64 and args.outer == "f64" and args.prec != "f64":
        supplement(line, "outer_df64", lambda: measure_outer_df64(args, cfg, dev, stream, rank, world, U_np, tune,
                                                                  ref_ln=ref_ln))
    if not args.no_tol_block and args.prec != "f64":
        # Dirichlet solves of the Schur pieces and the filter to 1e-10 instead of 1e-12
        supplement(line, "tol_block_1e-10", lambda: measure_outer_df64(
            args, cfg, dev, stream, rank, world, U_np, tune, outer=api.DD_PREC_F64, tol_block=1e-10, ref_ln=ref_ln))
    if not args.no_f32_storage and args.prec == "f16":
        # FP32 instead of FP16 storage of the inner solvers' vectors and links,
        # each inner solve reducing the residual by 1e-6 (two FP64 cycles)
        supplement(line, "inner_f32_storage", lambda: dict(measure_outer_df64(
            args, cfg, dev, stream, rank, world, U_np, tune, outer=api.DD_PREC_F64, ref_ln=ref_ln,
            prec=api.DD_PREC_F32, tol_inner=1e-6), tol_inner=1e-6))
    if not args.no_sap and args.prec != "f64":
        # the global solves by SAP-preconditioned flexible GCR instead of BiCGStab
        sap = {"sap_ncy": args.sap_ncy, "sap_nmr": args.sap_nmr, "sap_nkv": args.sap_nkv}
        supplement(line, "sap_gcr", lambda: dict(
            measure_outer_df64(args, cfg, dev, stream, rank, world, U_np, tune, krylov=api.DD_KRYLOV_SAP_GCR,
                               outer=api.DD_PREC_F64, sap=sap, ref_ln=ref_ln),
            parameters=sap, bicgstab_global_solves=iterations.get("global")))
    if args.compare_config:
        # mixed versus plain FP64 on smaller workloads (the FP64 path at the
        # full volume would hold the GPU for minutes per step)
        supplement(line, "mixed_vs_fp64", lambda: {name: compare_precisions(args, CONFIGS[name], dev, stream, rank)
                                                   for name in args.compare_config.split(",") if name})
    if not args.no_batched_filter:
        supplement(line, "batched_filter", lambda: measure_batched_filter(dev, stream))
    if not args.no_recursive:
        supplement(line, "recursive", lambda: measure_recursive(cfg, dev, stream))
    if not args.no_lu:
        supplement(line, "exact_lu", lambda: measure_lu(dev, stream))
    if rank == 0 and not args.no_cpu_baseline:
        c2 = CONFIGS["c2"]
        r = oracle_estimate_rate(c2)
        per_app, n, t = oracle_sample(cfg, seconds=15.0)
        line["cpu_baseline"] = {
            "value": r["all_cores"], "unit": "estimates/s", "cores": r["cores"], "kind": "oracle",
            "projected": False, "cpu": cpu_model(), "nproc": os.cpu_count(),
            "one_thread": r["one_thread"],
            "workload": "c2: 8^4 lattice, 4^4 blocks (active set of Sec. 3), eps 0.3, kappa 0.13, 16 factors",
            "sample": f"numpy FP64 oracle, whole global estimate of c2 (Schur pieces + global solve, delta form, "
                      f"every solve to relative residual 1e-10; proposal made before timing): factor 0 alone on "
                      f"one thread {r['seconds_one_factor']:.1f} s; all {r['factors']} factors, one process per "
                      f"core on {r['cores']} cores, {r['seconds_all_factors']:.1f} s",
            "gpu_same_workload": (line.get("mixed_vs_fp64") or {}).get("c2"),
            "c5_projection": {
                "value": 1.0 / (max(D_apps_per_est, 1e-9) * per_app), "unit": "estimates/s", "cores": 1,
                "projected": True,
                "sample": f"numpy FP64 oracle apply_D at V={V}: {n} applications in {t:.1f} s, scaled by "
                          f"{D_apps_per_est:.0f} Wilson applications per estimate measured on this run "
                          f"(global, Dirichlet and block-solver applications)"}}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def supplement(line, key, fn):
    """line[key] = fn(); an exception (a CUDA or library error of that one
    measurement) is printed to stderr and recorded as line[key] = {"error":
    ...}, so that the headline numbers measured before it are still printed."""
    import traceback
    try:
        line[key] = fn()
    except Exception as e:  # noqa: BLE001 - recorded, not hidden
        traceback.print_exc()
        line[key] = {"error": f"{type(e).__name__}: {e}"}


def measure_outer_df64(args, cfg, dev, stream, rank, world, U_np, tune, krylov=None, outer=None, sap=None,
                       tol_block=1e-12, ref_ln=None, prec=None, tol_inner=None):
    """The timed step again with the defect-correction residual in
    double-float arithmetic (outer_prec DD_PREC_DF64), or with another inner
    Krylov method (krylov, sap: DD_KRYLOV_SAP_GCR and its parameters), same
    workload, seeds and launch shapes; the hop kernels of the residual timed
    by kind, the iterations of the global solves counted."""
    import torch
    from paper_1112_1243_gb300 import api
    from paper_1112_1243_gb300.chain import HierarchicalStep
    prec = {"f16": api.DD_PREC_F16, "f32": api.DD_PREC_F32}[args.prec] if prec is None else prec
    tol_inner = args.tol_inner if tol_inner is None else tol_inner
    if krylov is None:
        krylov = {"cgnr": api.DD_KRYLOV_CGNR, "bicgstab": api.DD_KRYLOV_BICGSTAB,
                  "sap": api.DD_KRYLOV_SAP_GCR}[args.krylov]
    outer = api.DD_PREC_DF64 if outer is None else outer
    nmax = max(cfg["n_global"], cfg["n_block"])
    h = api.dd_init(cfg["dims"], cfg["block"], cfg["kappa"], max_rhs=nmax, inner_prec=prec,
                    block_prec=api.DD_PREC_F32, tol_global=1e-10, tol_block=tol_block, tol_inner=tol_inner,
                    maxit=40000, stream=stream, device=dev, krylov=krylov, outer_prec=outer, **(sap or {}))
    if tune:
        api.dd_set_tuning(h, hop_tpb=tune["hop_tpb"], hop_spt=tune["hop_spt"], hop64_tpb=tune["hop64_tpb"],
                          hop64_spt=tune["hop64_spt"], block_tpb=tune["block_tpb"],
                          block_ctas_per_sm=tune["block_ctas_per_sm"], filter_masked=tune["filter_masked"])
    U = torch.from_numpy(U_np).to(dev)
    chain = HierarchicalStep(h, BETA, n_inner=1, n_block=cfg["n_block"], n_global=cfg["n_global"],
                             seed=replica_seeds(cfg, rank)[1])
    for k in range(args.warmup):
        chain.step(U, k)
    torch.cuda.synchronize(dev)
    api.dd_kernel_timer(h, 1, 0, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lns = []
    for k in range(args.steps):
        ln, _ = chain.step(U, args.warmup + k)
        lns.append(ln.clone())
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms3, cnt3, _ = api.dd_kernel_timer(h, 2, 3)
    glob = api.dd_solver_stats(h, 0)
    diri = api.dd_solver_stats(h, 1)
    api.dd_kernel_timer(h, 0, 0)
    out = {"value": job_rate(cfg["n_global"] * args.steps, world, t_ms), "unit": "estimates/s",
           "ms_per_step": t_ms / args.steps, "device_status": api.dd_status(h)[0],
           "global_solves": dict(glob, inner_per_system=glob["inner_iterations"] / max(1, glob["systems"]),
                                 outer_cycles_per_solve=glob["outer_cycles"] / max(1, glob["solves"])),
           "dirichlet_solves": dict(diri, inner_per_system=diri["inner_iterations"] / max(1, diri["systems"]),
                                    outer_cycles_per_solve=diri["outer_cycles"] / max(1, diri["solves"]))}
    if cnt3:
        out.update(residual_hop_avg_us=1e3 * ms3 / max(1, cnt3), residual_hop_launches_timed=cnt3)
    if ref_ln is not None:
        # the same steps (field, seeds, step indices) as the default run: the
        # largest change of any ln r_i against it
        out["max_abs_dln_vs_default"] = max(float((a - b).abs().max()) for a, b in zip(lns, ref_ln))
        out["ln_scale"] = max(float(b.abs().max()) for b in ref_ln)
    del chain
    del h
    torch.cuda.empty_cache()
    return out


def compare_precisions(args, cfg, dev, stream, rank):
    """Estimates/s of the same hierarchical step with the mixed FP16/FP32 inner
    solvers and with the plain FP64 solver (CGNR), 3 warm-up + 2 timed steps each."""
    import torch
    from paper_1112_1243_gb300 import api, synthetic
    from paper_1112_1243_gb300.chain import HierarchicalStep
    out = {"workload": f"{'x'.join(map(str, cfg['dims']))} lattice, {'x'.join(map(str, cfg['block']))} blocks, "
                       f"kappa {cfg['kappa']}, eps {cfg['eps']}, {cfg['n_global']} global factors"}
    U_np = synthetic.random_gauge(cfg["dims"], cfg["eps"], replica_seeds(cfg, rank)[0])
    nmax = max(cfg["n_global"], cfg["n_block"])
    for name, prec, kry in (("mixed", api.DD_PREC_F16, api.DD_KRYLOV_BICGSTAB if args.krylov == "bicgstab"
                              else api.DD_KRYLOV_CGNR), ("fp64", api.DD_PREC_F64, api.DD_KRYLOV_CGNR)):
        h = api.dd_init(cfg["dims"], cfg["block"], cfg["kappa"], max_rhs=nmax, inner_prec=prec,
                        block_prec=api.DD_PREC_F32 if prec != api.DD_PREC_F64 else api.DD_PREC_F64,
                        tol_global=1e-10, tol_block=1e-12, maxit=40000, stream=stream, device=dev, krylov=kry)
        st = HierarchicalStep(h, BETA, n_inner=1, n_block=cfg["n_block"], n_global=cfg["n_global"],
                              seed=replica_seeds(cfg, rank)[1])
        U = torch.from_numpy(U_np).to(dev)
        for k in range(3):
            st.step(U, k)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(2):
            st.step(U, 3 + k)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        out[name] = cfg["n_global"] * 2 / (e0.elapsed_time(e1) / 1e3)
        del st
        del h
        torch.cuda.empty_cache()
    out["speedup"] = out["mixed"] / out["fp64"]
    return out


C4_LATTICES = [((16, 16, 16, 16), (4, 4, 4, 4)), ((12, 12, 12, 12), (6, 6, 6, 6)), ((16, 16, 16, 16), (8, 8, 8, 8))]


def measure_batched_filter(dev, stream, reps=3):
    """Block filters of three lattices with uneven blocks (256 x 4^4, 16 x 6^4,
    16 x 8^4; kappa 0.13, eps 0.3, 4 noise vectors per block) in one persistent
    launch per call: (block, factor) estimates per second."""
    import torch
    from paper_1112_1243_gb300 import api, synthetic
    n = 4
    hs, Us, Ups = [], [], []
    for k, (dims, block) in enumerate(C4_LATTICES):
        h = api.dd_init(dims, block, 0.13, max_rhs=n, stream=stream, device=dev)
        U = torch.from_numpy(synthetic.random_gauge(dims, 0.3, 4 + 10 * k)).to(dev)
        Up = U.clone()
        api.dd_gauge_update(h, Up, 3, BETA, 1, 0, 4, 1)
        hs.append(h)
        Us.append(U)
        Ups.append(Up)
    items = sum(h.nblocks for h in hs) * n
    work = [u.clone() for u in Ups]

    def one_call(ctr):
        for w, u in zip(work, Ups):
            w.copy_(u)
        api.dd_block_filter_batch(hs, Us, work, 3, n, 4, ctr)

    # launch shape of the persistent block solver for this mix of block sizes:
    # the candidates of the autotuner, each timed on one batch call
    best = None
    for tpb, ctas in ((256, 2), (256, 1), (128, 4), (128, 2)):
        for h in hs:
            api.dd_set_tuning(h, block_tpb=tpb, block_ctas_per_sm=ctas)
        one_call(1)
        torch.cuda.synchronize(dev)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        one_call(1)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        ms = c0.elapsed_time(c1)
        if best is None or ms < best[0]:
            best = (ms, tpb, ctas)
    for h in hs:
        api.dd_set_tuning(h, block_tpb=best[1], block_ctas_per_sm=best[2])
    tune = {"block_tpb": best[1], "block_ctas_per_sm": best[2]}
    for _ in range(2):
        for w, u in zip(work, Ups):
            w.copy_(u)
        api.dd_block_filter_batch(hs, Us, work, 3, n, 4, 2)
    torch.cuda.synchronize(dev)
    # the persistent launch timed with CUDA events on the first handle's
    # stream, with the kernel's own counts of inner iterations
    api.dd_kernel_timer(hs[0], 1, 0, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for r in range(reps):
        for w, u in zip(work, Ups):
            w.copy_(u)
        api.dd_block_filter_batch(hs, Us, work, 3, n, 4, 3 + r)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t = e0.elapsed_time(e1) / 1e3 / reps
    ms7, cnt7, _ = api.dd_kernel_timer(hs[0], 2, 7)
    st = api.dd_solver_stats(hs[0], 2)
    api.dd_kernel_timer(hs[0], 0, 0)
    # the same call recorded once as a CUDA graph on the first handle and replayed
    ln = [torch.zeros(h.nblocks, dtype=torch.float64, device=dev) for h in hs]
    acc = [torch.zeros(h.nblocks, dtype=torch.uint8, device=dev) for h in hs]
    for w, u in zip(work, Ups):
        w.copy_(u)
    api.dd_block_filter_batch(hs, Us, work, 3, n, 4, 3, ln, acc)
    for w, u in zip(work, Ups):
        w.copy_(u)
    api.dd_graph_begin(hs[0])
    try:
        api.dd_block_filter_batch(hs, Us, work, 3, n, 4, 3, ln, acc)
    finally:
        g = api.dd_graph_end(hs[0])
    for _ in range(2):
        for w, u in zip(work, Ups):
            w.copy_(u)
        api.dd_graph_launch(g, 0)
    torch.cuda.synchronize(dev)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for r in range(reps):
        for w, u in zip(work, Ups):
            w.copy_(u)
        api.dd_graph_launch(g, (r + 1) << 20)
    g1.record(stream)
    torch.cuda.synchronize(dev)
    tg = g0.elapsed_time(g1) / 1e3 / reps
    graph = {"seconds_per_call": tg, "block_estimates_per_s": items / tg, "top_level_nodes": api.dd_graph_nodes(g),
             "device_status": api.dd_status(hs[0])[0]}
    api.dd_graph_destroy(g)
    del g
    alu = peaks_alu(stream)
    kmodel = kernel_models((8, 8, 8, 8))[7]
    roof = roofline_entry(7, kmodel, ms7, cnt7, st["site_iterations"], 1e3 * t * reps, 6800.0, alu[0], alu[1])
    out = {"workload": "256 x 4^4 (16^4), 16 x 6^4 (12^4), 16 x 8^4 (16^4) blocks, 4 noise vectors each, "
                       "one persistent launch", "items_per_launch": items, "seconds_per_call": t,
           "block_estimates_per_s": items / t,
           "launch_shape": {"threads": tune["block_tpb"], "blocks_per_sm": tune["block_ctas_per_sm"]},
           "iterations": dict(st, inner_per_item=st["inner_iterations"] / max(1, st["items"]),
                              outer_per_item=st["outer_cycles"] / max(1, st["items"])),
           "roofline": roof, "graph": graph}
    for h in hs:
        del h
    return out


def measure_lu(dev, stream, reps=3):
    """The exact check path on the 4^4 lattice with 2^4 blocks (c1): ln|det|
    of D (3072 x 3072 complex), of the 16 Dirichlet blocks (192 x 192) and
    of the Schur complement (1536 x 1536, assembled with block solves and a
    product), by dense LU with partial pivoting; CUDA-event time per call and
    the FP64 rate of the full-matrix LU (8 n^3 / 3 real flops)."""
    import torch
    from paper_1112_1243_gb300 import api, synthetic
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    h = api.dd_init(dims, block, 0.12, features=api.DD_FEAT_EXACT, stream=stream, device=dev)
    U = torch.from_numpy(synthetic.random_gauge(dims, 0.4, 1)).to(dev)
    out = {"workload": "c1: 4^4 lattice, 2^4 blocks, kappa 0.12, eps 0.4"}
    alu, src = peaks_alu(stream)
    for which, name, n, nmat, tc in ((0, "D", 3072, 1, True), (1, "D_b", 192, 16, True), (2, "Dhat", 1536, 1, True),
                                     (0, "D_fp64_update", 3072, 1, False), (2, "Dhat_fp64_update", 1536, 1, False)):
        api.dd_lu_tensor_cores(h, tc)
        api.dd_logdet_exact(h, U, which)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            api.dd_logdet_exact(h, U, which)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": ms, "n": n, "matrices": nmat}
        out[name]["trailing_update"] = ("FP16 tensor cores (Ozaki slices, FP64 accuracy)" if tc and n > 384
                                        else "FP64 FMA")
        if which == 0:
            tf = 8.0 * n ** 3 / 3.0 / (ms / 1e3) / 1e12
            out[name].update(achieved_tflops=tf, peak_fp64_tflops=alu["fp64_fma"], frac=tf / alu["fp64_fma"],
                             peak_fp64_mma_tflops=alu["fp64_mma"], peak_source=src)
    del h
    return out


def measure_recursive(cfg, dev, stream, n_schur=4, steps=1):
    """The benchmark step with one level of recursion (Eq. 4step steps 0-3):
    the blocks of the workload split into 4^4 sub-blocks, step 1 on the
    sub-blocks, step 2 (the blocks' Schur complements, n_schur factors) on
    the blocks, then the global step; global estimates per second."""
    import torch
    from paper_1112_1243_gb300 import api, synthetic
    from paper_1112_1243_gb300.chain import HierarchicalStep
    sub = tuple(b // 2 for b in cfg["block"])
    nmax = max(cfg["n_global"], cfg["n_block"], n_schur)
    h = api.dd_init(cfg["dims"], cfg["block"], cfg["kappa"], max_rhs=nmax, inner_prec=api.DD_PREC_F16,
                    tol_global=1e-10, tol_block=1e-12, tol_inner=1e-3, maxit=40000, stream=stream, device=dev,
                    krylov=api.DD_KRYLOV_BICGSTAB, sub_block=sub)
    U = torch.from_numpy(synthetic.random_gauge(cfg["dims"], cfg["eps"], cfg["seed"])).to(dev)
    chain = HierarchicalStep(h, BETA, n_inner=1, n_block=cfg["n_block"], n_global=cfg["n_global"],
                             seed=cfg["seed"] * 7919, n_schur=n_schur)
    chain.step(U, 0)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        chain.step(U, 1 + k)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t = e0.elapsed_time(e1) / 1e3 / steps
    out = {"workload": f"{'x'.join(map(str, cfg['dims']))} lattice, {'x'.join(map(str, cfg['block']))} blocks "
                       f"split into {'x'.join(map(str, sub))} sub-blocks (active links of the sub-blocks), "
                       f"{cfg['n_block']} sub-block, {n_schur} block-Schur and {cfg['n_global']} global factors",
           "value": cfg["n_global"] / t, "unit": "estimates/s", "ms_per_step": 1e3 * t,
           "block_schur_accept_rate_last_step": float(chain.acc_bs.float().mean().item()),
           "sub_block_accept_rate_last_step": float(chain.acc_b.float().mean().item()),
           "device_status": api.dd_status(h)[0]}
    del chain
    del h
    torch.cuda.empty_cache()
    return out


def run_solve(args, cfg):
    """Global solves D x = b (one right-hand side) on a handle planned for
    solves only: the hop kernels of the hot path at a few GB of device memory."""
    import torch
    from paper_1112_1243_gb300 import api, build, synthetic
    build.build()
    dev = torch.device("cuda", 0)
    prec = {"f16": api.DD_PREC_F16, "f32": api.DD_PREC_F32, "f64": api.DD_PREC_F64}[args.prec]
    krylov = {"cgnr": api.DD_KRYLOV_CGNR, "bicgstab": api.DD_KRYLOV_BICGSTAB, "sap": api.DD_KRYLOV_SAP_GCR}[args.krylov]
    outer = {"f64": api.DD_PREC_F64, "df64": api.DD_PREC_DF64}[args.outer]
    h = api.dd_init(cfg["dims"], cfg["block"], cfg["kappa"], max_rhs=1, inner_prec=prec, tol_global=1e-10,
                    tol_inner=args.tol_inner, maxit=40000, features=api.DD_FEAT_SOLVE, device=dev, krylov=krylov,
                    outer_prec=outer, sap_ncy=args.sap_ncy, sap_nmr=args.sap_nmr, sap_nkv=args.sap_nkv)
    U = torch.from_numpy(synthetic.random_gauge(cfg["dims"], cfg["eps"], cfg["seed"])).to(dev)
    b = torch.from_numpy(synthetic.random_spinor(cfg["dims"], 1)).to(dev)
    x = torch.zeros_like(b)
    for _ in range(args.warmup):
        api.dd_solve(h, x, b, U, 1, prec)
    torch.cuda.synchronize()
    api.dd_kernel_timer(h, 1, 0, 1)
    t0 = time.perf_counter()
    its = 0
    for _ in range(args.steps):
        it, res, _ = api.dd_solve(h, x, b, U, 1, prec)
        its += it
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    st = api.dd_solver_stats(h, 0)
    out = {"mode": "solve", "config": args.config, "prec": args.prec, "outer": args.outer,
           "tol_inner": args.tol_inner, "seconds_per_solve": t / args.steps,
           "inner_iterations_per_solve": its / args.steps, "relres": res[0],
           "outer_cycles_per_solve": st["outer_cycles"] / max(1, st["solves"])}
    for kind in (0, 1, 2, 3):
        ms, cnt, sites = api.dd_kernel_timer(h, 2, kind)
        if cnt:
            out[f"hop_kind{kind}"] = {"launches": cnt, "avg_us": 1e3 * ms / cnt,
                                      "GB_per_s": sites * HOP_BYTES[kind] / 1e9 / (ms / 1e3)}
    print(json.dumps(out))
    return 0


def main():
    args = parse()
    cfg = CONFIGS[args.config]
    if args.impl == "reference":
        return run_reference(args, cfg)
    if args.mode == "solve":
        return run_solve(args, cfg)
    if args.mode == "lu":
        import torch
        from paper_1112_1243_gb300 import build
        build.build()
        dev = torch.device("cuda", 0)
        print(json.dumps({"mode": "lu", "exact_lu": measure_lu(dev, torch.cuda.current_stream(dev))}))
        return 0
    return run_gpu(args, cfg)


if __name__ == "__main__":
    sys.exit(main())
