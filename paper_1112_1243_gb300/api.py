"""Python binding of the C ABI (include/dd.h) with the same entry-point names.

Device buffers are torch tensors (PyTorch provides device memory and the
stream); every function here only marshals arguments and calls libdd.so.
Fields use the canonical FP64 layouts of the C ABI:
  gauge field  complex128 tensor of shape (V, 4, 3, 3)
  spinors      complex128 tensor of shape (nrhs, V, 4, 3) or (V, 4, 3)
"""
import ctypes

import torch

from . import _lib
from ._lib import *  # noqa: F401,F403  (constants)


class DDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_lib.ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Handle:
    """A dd_t handle plus the torch-owned workspace it uses."""

    def __init__(self, ptr, params, workspace, stream):
        self.ptr = ptr
        self.params = params
        self.workspace = workspace
        self.stream = stream
        self.dims = tuple(params.dims)
        self.block = tuple(params.block)
        self.V = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]
        self.nblocks = 1
        for L, b in zip(self.dims, self.block):
            self.nblocks *= L // b
        self.sub_block = tuple(params.sub_block) if any(params.sub_block) else None
        # blocks of the smallest level (the block filter's blocks)
        self.nfine = 1
        for L, b in zip(self.dims, self.sub_block or self.block):
            self.nfine *= L // b

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                _lib.load().dd_finalize(self.ptr)
            except Exception:
                pass
            self.ptr = None


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensors passed to the library must be contiguous")
    return t.data_ptr()


def _check(h, rc):
    if rc != _lib.DD_OK:
        lib = _lib.load()
        msg = lib.dd_last_error(h.ptr if isinstance(h, Handle) else h)
        raise DDError(rc, msg.decode() if msg else "")
    return rc


def dd_default_params():
    p = _lib.dd_params()
    _lib.load().dd_default_params(ctypes.byref(p))
    return p


def dd_init(dims, block, kappa, bc_time=-1, active_mode=_lib.DD_ACTIVE_AUTO, max_rhs=1,
            inner_prec=_lib.DD_PREC_F16, block_prec=_lib.DD_PREC_F32, tol_global=1e-10,
            tol_block=1e-12, tol_inner=1e-3, maxit=20000, stream=None, device=None, features=0,
            krylov=_lib.DD_KRYLOV_CGNR, sub_block=None, outer_prec=_lib.DD_PREC_F64, sap_ncy=None, sap_nmr=None,
            sap_nkv=None):
    """Create a handle and give it a torch-allocated workspace on `device`.
    sub_block: extents of the sub-blocks of one level of recursion (None: no
    recursion).  outer_prec: arithmetic of the defect-correction residual of
    mixed-precision solves (DD_PREC_F64 or DD_PREC_DF64)."""
    lib = _lib.load()
    p = dd_default_params()
    for a in range(4):
        p.dims[a] = int(dims[a])
        p.block[a] = int(block[a])
    p.kappa = float(kappa)
    p.bc_time = int(bc_time)
    p.active_mode = int(active_mode)
    p.max_rhs = int(max_rhs)
    p.inner_prec = int(inner_prec)
    p.block_prec = int(block_prec)
    p.tol_global = float(tol_global)
    p.tol_block = float(tol_block)
    p.tol_inner = float(tol_inner)
    p.maxit = int(maxit)
    p.features = int(features)
    p.krylov = int(krylov)
    for a in range(4):
        p.sub_block[a] = int(sub_block[a]) if sub_block is not None else 0
    p.outer_prec = int(outer_prec)
    if sap_ncy is not None:
        p.sap_ncy = int(sap_ncy)
    if sap_nmr is not None:
        p.sap_nmr = int(sap_nmr)
    if sap_nkv is not None:
        p.sap_nkv = int(sap_nkv)
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if stream is None:
        stream = torch.cuda.current_stream(device)
    h = ctypes.c_void_p()
    rc = lib.dd_init(ctypes.byref(h), ctypes.byref(p), ctypes.c_void_p(stream.cuda_stream))
    if rc != _lib.DD_OK:
        raise DDError(rc, "dd_init failed (check extents, blocks and parameters)")
    size = ctypes.c_size_t()
    _check(h, lib.dd_workspace_size(h, ctypes.byref(size)))
    ws = torch.empty(size.value + 256, dtype=torch.uint8, device=device)
    base = (ws.data_ptr() + 255) & ~255
    _check(h, lib.dd_set_workspace(h, ctypes.c_void_p(base), ctypes.c_size_t(size.value)))
    return Handle(h, p, ws, stream)


def dd_get_maps(h):
    """Host copies of the geometry tables as numpy arrays."""
    import numpy as np
    V = h.V
    nbr = np.zeros(V * 8, dtype=np.int32)
    sign = np.zeros(V * 8, dtype=np.int32)
    order = np.zeros(V, dtype=np.int32)
    blk = np.zeros(V, dtype=np.int32)
    act = np.zeros(V * 4, dtype=np.uint8)
    _check(h, _lib.load().dd_get_maps(h.ptr, nbr.ctypes.data, sign.ctypes.data, order.ctypes.data,
                                      blk.ctypes.data, act.ctypes.data))
    return {"nbr": nbr.reshape(V, 4, 2), "sign": sign.reshape(V, 4, 2), "dd_order": order,
            "block_of": blk, "active": act.reshape(V, 4).astype(bool)}


def dd_apply_D(h, out, inp, U, op=_lib.DD_OP_D, prec=_lib.DD_PREC_F64, nrhs=1):
    return _check(h, _lib.load().dd_apply_D(h.ptr, _ptr(out), _ptr(inp), _ptr(U), int(op), int(prec), int(nrhs)))


def dd_apply_D_block(h, out, inp, U, colour_mask=3, prec=_lib.DD_PREC_F64, nrhs=1):
    return _check(h, _lib.load().dd_apply_D_block(h.ptr, _ptr(out), _ptr(inp), _ptr(U), int(colour_mask),
                                                  int(prec), int(nrhs)))


def dd_solve(h, x, b, U, nrhs=1, prec=_lib.DD_PREC_F64, check=True):
    """Returns (total inner iterations, list of true relative residuals, rc)."""
    import numpy as np
    it = ctypes.c_int(0)
    res = np.zeros(max(1, nrhs), dtype=np.float64)
    rc = _lib.load().dd_solve(h.ptr, _ptr(x), _ptr(b), _ptr(U), int(nrhs), int(prec), ctypes.byref(it),
                              res.ctypes.data)
    if check:
        _check(h, rc)
    return it.value, res.tolist(), rc


def dd_sap_apply(h, out, inp, U, nrhs=1, prec=_lib.DD_PREC_F32):
    """sap_ncy Schwarz cycles (the SAP-GCR preconditioner) applied to inp."""
    return _check(h, _lib.load().dd_sap_apply(h.ptr, _ptr(out), _ptr(inp), _ptr(U), int(nrhs), int(prec)))


def dd_noise(h, eta, nrhs, purpose, seed, ctr):
    return _check(h, _lib.load().dd_noise(h.ptr, _ptr(eta), int(nrhs), int(purpose), int(seed), int(ctr)))


def dd_interpolate(h, Ut, U, Unew, i, n):
    return _check(h, _lib.load().dd_interpolate(h.ptr, _ptr(Ut), _ptr(U), _ptr(Unew), int(i), int(n)))


def dd_det_ratio_estimate(h, U_old, U_new, n, seed, ctr, mode=_lib.DD_EST_FACTORS, ln_out=None):
    if ln_out is None:
        ln_out = torch.zeros(n, dtype=torch.float64, device=h.workspace.device)
    _check(h, _lib.load().dd_det_ratio_estimate(h.ptr, _ptr(U_old), _ptr(U_new), int(n), int(seed), int(ctr),
                                                int(mode), _ptr(ln_out)))
    return ln_out


def dd_block_filter(h, U_old, U_new, colour_mask, mode, n, seed, ctr, ln_b=None, accept=None):
    dev = h.workspace.device
    if ln_b is None:
        ln_b = torch.zeros(h.nfine, dtype=torch.float64, device=dev)
    if accept is None:
        accept = torch.zeros(h.nfine, dtype=torch.uint8, device=dev)
    _check(h, _lib.load().dd_block_filter(h.ptr, _ptr(U_old), _ptr(U_new), int(colour_mask), int(mode), int(n),
                                          int(seed), int(ctr), _ptr(ln_b), _ptr(accept)))
    return ln_b, accept


def dd_block_schur_filter(h, U_old, U_new, colour_mask, n, seed, ctr, ln_b=None, accept=None):
    """Step 2 of the hierarchy (handles with sub-blocks): per-block Schur
    log-ratios over the blocks, decisions, restore."""
    dev = h.workspace.device
    if ln_b is None:
        ln_b = torch.zeros(h.nblocks, dtype=torch.float64, device=dev)
    if accept is None:
        accept = torch.zeros(h.nblocks, dtype=torch.uint8, device=dev)
    _check(h, _lib.load().dd_block_schur_filter(h.ptr, _ptr(U_old), _ptr(U_new), int(colour_mask), int(n),
                                                int(seed), int(ctr), _ptr(ln_b), _ptr(accept)))
    return ln_b, accept


def dd_relative_gauge_fix(h, U, U_new, sweeps, functional=None):
    """U_new <- U_new^g with g raising sum Re tr(U^dag g U_new g^dag) (in place)."""
    return _check(h, _lib.load().dd_relative_gauge_fix(h.ptr, _ptr(U), _ptr(U_new), int(sweeps), _ptr(functional)))


def dd_block_filter_batch(hs, U_olds, U_news, colour_mask, n, seed, ctr, ln_bs=None, accepts=None):
    """Block filters of several handles (lattices, block shapes) in one persistent launch."""
    lib = _lib.load()
    nh = len(hs)
    dev = hs[0].workspace.device
    harr = (ctypes.c_void_p * nh)(*[h.ptr.value if isinstance(h.ptr, ctypes.c_void_p) else h.ptr for h in hs])
    size = ctypes.c_size_t()
    rc = lib.dd_block_filter_batch_workspace(nh, harr, int(n), ctypes.byref(size))
    if rc != _lib.DD_OK:
        raise DDError(rc, "dd_block_filter_batch_workspace failed")
    # the scratch of the last call is reused when large enough (a CUDA-graph
    # capture of this call needs the scratch of the eager call before it)
    ws = getattr(hs[0], "batch_ws", None)
    if ws is None or ws.numel() < size.value + 256 or ws.device != dev:
        ws = torch.empty(size.value + 256, dtype=torch.uint8, device=dev)
    base = (ws.data_ptr() + 255) & ~255
    if ln_bs is None:
        ln_bs = [torch.zeros(h.nblocks, dtype=torch.float64, device=dev) for h in hs]
    if accepts is None:
        accepts = [torch.zeros(h.nblocks, dtype=torch.uint8, device=dev) for h in hs]
    arr = lambda ts: (ctypes.c_void_p * nh)(*[_ptr(t) for t in ts])
    rc = lib.dd_block_filter_batch(nh, harr, arr(U_olds), arr(U_news), int(colour_mask), int(n), int(seed), int(ctr),
                                   arr(ln_bs), arr(accepts), ctypes.c_void_p(base), ctypes.c_size_t(size.value))
    if rc != _lib.DD_OK:
        raise DDError(rc, dd_last_error(hs[0]))
    hs[0].batch_ws = ws  # keep the scratch alive until the stream has consumed it
    return ln_bs, accepts


def dd_gauge_update(h, U, colour_mask, beta, n_hb, n_or, seed, ctr):
    return _check(h, _lib.load().dd_gauge_update(h.ptr, _ptr(U), int(colour_mask), float(beta), int(n_hb),
                                                 int(n_or), int(seed), int(ctr)))


def dd_global_accept(h, U, U_old, ln_r, seed, ctr, accept=None, margin=None):
    dev = h.workspace.device
    if accept is None:
        accept = torch.zeros(1, dtype=torch.uint8, device=dev)
    if margin is None:
        margin = torch.zeros(1, dtype=torch.float64, device=dev)
    _check(h, _lib.load().dd_global_accept(h.ptr, _ptr(U), _ptr(U_old), _ptr(ln_r), int(ln_r.numel()), int(seed),
                                           int(ctr), _ptr(accept), _ptr(margin)))
    return accept, margin


def dd_logdet_exact(h, U, which, out=None):
    if out is None:
        n = h.nblocks if which == 1 else 1
        out = torch.zeros(n, dtype=torch.float64, device=h.workspace.device)
    _check(h, _lib.load().dd_logdet_exact(h.ptr, _ptr(U), int(which), _ptr(out)))
    return out


def dd_plaquette(h, U, out=None):
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device=h.workspace.device)
    _check(h, _lib.load().dd_plaquette(h.ptr, _ptr(U), _ptr(out)))
    return out


def dd_sync(h):
    return _check(h, _lib.load().dd_sync(h.ptr))


def dd_status(h):
    st = ctypes.c_int(0)
    hb = ctypes.c_longlong(0)
    _check(h, _lib.load().dd_status(h.ptr, ctypes.byref(st), ctypes.byref(hb)))
    return st.value, hb.value


def dd_last_error(h):
    m = _lib.load().dd_last_error(h.ptr)
    return m.decode() if m else ""


def dd_launch_count(h):
    n = ctypes.c_longlong(0)
    _check(h, _lib.load().dd_launch_count(h.ptr, ctypes.byref(n)))
    return n.value


def dd_kernel_timer(h, op, kind=0, every=1):
    """op 1: start, 0: stop, 2: read -> (total ms, timed launches, sites processed)."""
    ms = ctypes.c_double(0.0)
    cnt = ctypes.c_longlong(0)
    sites = ctypes.c_longlong(0)
    _check(h, _lib.load().dd_kernel_timer(h.ptr, int(op), int(kind), int(every), ctypes.byref(ms),
                                          ctypes.byref(cnt), ctypes.byref(sites)))
    return ms.value, cnt.value, sites.value


def dd_block_ratios_range(h, U_old, U_new, pos0, npos, n, seed, ctr, ln_b=None):
    """Stochastic block log-ratios of the blocks at block-order positions
    [pos0, pos0 + npos); 0 for the other blocks."""
    if ln_b is None:
        ln_b = torch.zeros(h.nfine, dtype=torch.float64, device=h.workspace.device)
    _check(h, _lib.load().dd_block_ratios_range(h.ptr, _ptr(U_old), _ptr(U_new), int(pos0), int(npos), int(n),
                                                int(seed), int(ctr), _ptr(ln_b)))
    return ln_b


def dd_block_accept(h, U_old, U_new, colour_mask, ln_b, seed, ctr, accept=None):
    """Block decisions from a complete ln_b and the restore of rejected blocks in U_new."""
    if accept is None:
        accept = torch.zeros(h.nfine, dtype=torch.uint8, device=h.workspace.device)
    _check(h, _lib.load().dd_block_accept(h.ptr, _ptr(U_old), _ptr(U_new), int(colour_mask), _ptr(ln_b), int(seed),
                                          int(ctr), _ptr(accept)))
    return accept


def dd_solver_stats(h, kind):
    """kind 0 whole-lattice solves, 1 Dirichlet solves, 2 persistent block
    solver -> dict of the counters since the last dd_kernel_timer(op 1)."""
    out = (ctypes.c_longlong * 5)()
    _check(h, _lib.load().dd_solver_stats(h.ptr, int(kind), out))
    names = ("solves", "systems", "inner_iterations", "outer_cycles", "site_iterations") if kind < 2 else \
        ("launches", "items", "inner_iterations", "outer_cycles", "site_iterations")
    return dict(zip(names, list(out)))


def dd_lu_tensor_cores(h, on=True):
    """Trailing update of the dense LU on the tensor cores (Ozaki slices with
    FP64 accuracy; default) or on the FP64 FMA pipe."""
    _check(h, _lib.load().dd_lu_tensor_cores(h.ptr, 1 if on else 0))


def dd_barrier_check(h, missing=0):
    """Grid barrier of the LU panel launch with `missing` arrivals that never
    come: True when every thread block passed (the bounded wait raises
    DD_ERR_TIMEOUT in the device status word otherwise)."""
    out = ctypes.c_int()
    _check(h, _lib.load().dd_barrier_check(h.ptr, int(missing), ctypes.byref(out)))
    return bool(out.value)


def dd_alu_peaks(stream=None):
    """Measured FP64 FMA, FP32 FMA and FP64 mma.sync throughput (TFLOP/s) of the current GPU."""
    out = (ctypes.c_double * 3)()
    s = (stream or torch.cuda.current_stream()).cuda_stream
    rc = _lib.load().dd_alu_peaks(out, ctypes.c_void_p(s))
    if rc != _lib.DD_OK:
        raise DDError(rc, "dd_alu_peaks failed")
    return {"fp64_fma": out[0], "fp32_fma": out[1], "fp64_mma": out[2]}


def dd_block_ratios_noalloc(dims, block, kappa, bc_time, colour_mask, U_old, U_new, seed, ctr, tol_block, ln_b,
                            stream=None):
    """Allocation-free one-factor block log-ratios (no handle, no workspace);
    ln_b is a caller-owned device tensor of nblocks doubles."""
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    b = (ctypes.c_int * 4)(*[int(v) for v in block])
    s = (stream or torch.cuda.current_stream()).cuda_stream
    rc = _lib.load().dd_block_ratios_noalloc(d, b, float(kappa), int(bc_time), int(colour_mask), _ptr(U_old),
                                             _ptr(U_new), int(seed), int(ctr), float(tol_block), _ptr(ln_b),
                                             ctypes.c_void_p(s))
    if rc != _lib.DD_OK:
        raise DDError(rc, "dd_block_ratios_noalloc failed")
    return ln_b


def dd_chain_step(h, U, params, buffers, step):
    """One hierarchical step on the device (U updated in place).  params: a
    _lib.dd_chain_params; buffers: dict of the device tensors U0, Up, ln_b,
    acc_b, ln_g, acc_g, margin."""
    bufs = _lib.dd_chain_buffers(*[_ptr(buffers.get(k)) for k in ("U0", "Up", "ln_b", "acc_b", "ln_g", "acc_g",
                                                                     "margin", "ln_bs", "acc_bs")])
    return _check(h, _lib.load().dd_chain_step(h.ptr, _ptr(U), ctypes.byref(params), ctypes.byref(bufs),
                                               int(step)))


class Graph:
    """An instantiated CUDA graph of library calls (dd_graph_t)."""

    def __init__(self, h, ptr):
        self.h = h
        self.ptr = ptr

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                _lib.load().dd_graph_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def dd_graph_begin(h):
    return _check(h, _lib.load().dd_graph_begin(h.ptr))


def dd_graph_end(h):
    g = ctypes.c_void_p()
    _check(h, _lib.load().dd_graph_end(h.ptr, ctypes.byref(g)))
    return Graph(h, g.value)


def dd_graph_launch(g, ctr_offset=0):
    return _check(g.h, _lib.load().dd_graph_launch(g.ptr, int(ctr_offset)))


def dd_graph_nodes(g):
    n = ctypes.c_size_t()
    _check(g.h, _lib.load().dd_graph_nodes(g.ptr, ctypes.byref(n)))
    return n.value


def dd_graph_destroy(g):
    if g.ptr:
        rc = _lib.load().dd_graph_destroy(g.ptr)
        g.ptr = None
        return rc
    return 0


def dd_autotune(h, what=_lib.DD_TUNE_HOP, U_old=None, U_new=None, reps=20):
    """Time the candidate launch shapes on this handle and keep the fastest;
    returns the report as a dict."""
    r = _lib.dd_tune_report()
    _check(h, _lib.load().dd_autotune(h.ptr, int(what), _ptr(U_old), _ptr(U_new), int(reps), ctypes.byref(r)))
    return {name: getattr(r, name) for name, _ in r._fields_}


def dd_set_tuning(h, hop_tpb=128, hop_spt=1, hop64_tpb=128, hop64_spt=1, block_tpb=256, block_ctas_per_sm=2,
                  filter_masked=0):
    return _check(h, _lib.load().dd_set_tuning(h.ptr, int(hop_tpb), int(hop_spt), int(hop64_tpb), int(hop64_spt),
                                               int(block_tpb), int(block_ctas_per_sm), int(filter_masked)))


def dd_finalize(h):
    if h.ptr:
        rc = _lib.load().dd_finalize(h.ptr)
        h.ptr = None
        return rc
    return 0
