"""ctypes binding of the C ABI declared in include/dd.h.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libdd.so.  The library is loaded from this package directory; if
it is missing the import fails loudly (there is no CPU fallback).
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdd.so")

DD_OK = 0
DD_ERR_INVALID_ARG = -1
DD_ERR_UNSUPPORTED = -2
DD_ERR_CUDA = -3
DD_ERR_NOT_CONVERGED = -4
DD_ERR_NUMERIC = -5
DD_ERR_TIMEOUT = -6
DD_ERR_NO_WORKSPACE = -7

DD_PREC_F64, DD_PREC_F32, DD_PREC_F16, DD_PREC_DF64 = 0, 1, 2, 3
DD_ACTIVE_AUTO, DD_ACTIVE_PAPER, DD_ACTIVE_INNER6, DD_ACTIVE_INTRA, DD_ACTIVE_ALL = 0, 1, 2, 3, 4
DD_OP_D, DD_OP_DDAG, DD_OP_DTILDE, DD_OP_DTILDE_DAG, DD_OP_HEO, DD_OP_INTER = 0, 1, 2, 3, 4, 5
DD_PURPOSE_GLOBAL_NOISE = 1
DD_PURPOSE_BLOCK_NOISE = 2
DD_PURPOSE_HEATBATH = 3
DD_PURPOSE_BLOCK_ACCEPT = 5
DD_PURPOSE_GLOBAL_ACCEPT = 6
DD_PURPOSE_USER_NOISE = 7
DD_PURPOSE_BLOCK_SCHUR_NOISE = 4
DD_PURPOSE_BLOCK_SCHUR_ACCEPT = 8
DD_EST_FACTORS, DD_EST_REPLICAS, DD_EST_INTERP_ALL = 0, 1, 4
DD_FILTER_STOCHASTIC, DD_FILTER_EXACT = 0, 1
DD_TIMER_KIND_COUNT = 10
DD_KRYLOV_CGNR, DD_KRYLOV_BICGSTAB, DD_KRYLOV_SAP_GCR = 0, 1, 2

ERROR_NAMES = {
    DD_ERR_INVALID_ARG: "DD_ERR_INVALID_ARG",
    DD_ERR_UNSUPPORTED: "DD_ERR_UNSUPPORTED",
    DD_ERR_CUDA: "DD_ERR_CUDA",
    DD_ERR_NOT_CONVERGED: "DD_ERR_NOT_CONVERGED",
    DD_ERR_NUMERIC: "DD_ERR_NUMERIC",
    DD_ERR_TIMEOUT: "DD_ERR_TIMEOUT",
    DD_ERR_NO_WORKSPACE: "DD_ERR_NO_WORKSPACE",
}


class dd_params(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int * 4),
        ("block", ctypes.c_int * 4),
        ("kappa", ctypes.c_double),
        ("bc_time", ctypes.c_int),
        ("active_mode", ctypes.c_int),
        ("max_rhs", ctypes.c_int),
        ("inner_prec", ctypes.c_int),
        ("block_prec", ctypes.c_int),
        ("tol_global", ctypes.c_double),
        ("tol_block", ctypes.c_double),
        ("tol_inner", ctypes.c_double),
        ("maxit", ctypes.c_int),
        ("features", ctypes.c_int),
        ("krylov", ctypes.c_int),
        ("sub_block", ctypes.c_int * 4),
        ("outer_prec", ctypes.c_int),
        ("sap_ncy", ctypes.c_int),
        ("sap_nmr", ctypes.c_int),
        ("sap_nkv", ctypes.c_int),
    ]


class dd_chain_params(ctypes.Structure):
    _fields_ = [
        ("beta", ctypes.c_double),
        ("n_inner", ctypes.c_int),
        ("n_block", ctypes.c_int),
        ("n_global", ctypes.c_int),
        ("n_hb", ctypes.c_int),
        ("n_or", ctypes.c_int),
        ("filter_mode", ctypes.c_int),
        ("colour_passes", ctypes.c_int),
        ("n_schur", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("gauge_fix_sweeps", ctypes.c_int),
        ("reserved", ctypes.c_int),
    ]


class dd_chain_buffers(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in ("U0", "Up", "ln_b", "acc_b", "ln_g", "acc_g", "margin",
                                                     "ln_bs", "acc_bs")]


class dd_tune_report(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("hop_tpb", "hop_spt", "hop64_tpb", "hop64_spt", "block_tpb",
                                              "block_ctas_per_sm", "from_cache")] + \
               [(n, ctypes.c_float) for n in ("hop_ms", "hop_default_ms", "hop64_ms", "hop64_default_ms", "block_ms",
                                              "block_default_ms")] + \
               [("filter_masked", ctypes.c_int), ("filter_masked_ms", ctypes.c_float)]


DD_TUNE_HOP, DD_TUNE_BLOCK, DD_TUNE_NO_CACHE = 1, 2, 4
DD_FEAT_SOLVE, DD_FEAT_ESTIMATE, DD_FEAT_EXACT = 1, 2, 4


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_U64 = ctypes.c_uint64

# name -> (argtypes); every function returns int except dd_last_error
SIGNATURES = {
    "dd_default_params": [ctypes.POINTER(dd_params)],
    "dd_init": [ctypes.POINTER(_P), ctypes.POINTER(dd_params), _P],
    "dd_workspace_size": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "dd_set_workspace": [_P, _P, ctypes.c_size_t],
    "dd_get_maps": [_P, _P, _P, _P, _P, _P],
    "dd_apply_D": [_P, _P, _P, _P, _I, _I, _I],
    "dd_apply_D_block": [_P, _P, _P, _P, _I, _I, _I],
    "dd_solve": [_P, _P, _P, _P, _I, _I, ctypes.POINTER(_I), _P],
    "dd_noise": [_P, _P, _I, _I, _U64, _U64],
    "dd_interpolate": [_P, _P, _P, _P, _I, _I],
    "dd_det_ratio_estimate": [_P, _P, _P, _I, _U64, _U64, _I, _P],
    "dd_block_filter": [_P, _P, _P, _I, _I, _I, _U64, _U64, _P, _P],
    "dd_block_schur_filter": [_P, _P, _P, _I, _I, _U64, _U64, _P, _P],
    "dd_relative_gauge_fix": [_P, _P, _P, _I, _P],
    "dd_block_filter_batch_workspace": [_I, _P, _I, ctypes.POINTER(ctypes.c_size_t)],
    "dd_block_filter_batch": [_I, _P, _P, _P, _I, _I, _U64, _U64, _P, _P, _P, ctypes.c_size_t],
    "dd_gauge_update": [_P, _P, _I, _D, _I, _I, _U64, _U64],
    "dd_global_accept": [_P, _P, _P, _P, _I, _U64, _U64, _P, _P],
    "dd_logdet_exact": [_P, _P, _I, _P],
    "dd_plaquette": [_P, _P, _P],
    "dd_sync": [_P],
    "dd_status": [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_longlong)],
    "dd_last_error": [_P],
    "dd_launch_count": [_P, ctypes.POINTER(ctypes.c_longlong)],
    "dd_kernel_timer": [_P, _I, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong),
                        ctypes.POINTER(ctypes.c_longlong)],
    "dd_solver_stats": [_P, _I, ctypes.POINTER(ctypes.c_longlong)],
    "dd_sap_apply": [_P, _P, _P, _P, _I, _I],
    "dd_block_ratios_range": [_P, _P, _P, _I, _I, _I, _U64, _U64, _P],
    "dd_block_accept": [_P, _P, _P, _I, _P, _U64, _U64, _P],
    "dd_alu_peaks": [ctypes.POINTER(_D), _P],
    "dd_barrier_check": [_P, _I, ctypes.POINTER(_I)],
    "dd_lu_tensor_cores": [_P, _I],
    "dd_block_ratios_noalloc": [ctypes.POINTER(_I), ctypes.POINTER(_I), _D, _I, _I, _P, _P, _U64, _U64, _D, _P,
                                _P],
    "dd_chain_step": [_P, _P, ctypes.POINTER(dd_chain_params), ctypes.POINTER(dd_chain_buffers), ctypes.c_ulonglong],
    "dd_graph_begin": [_P],
    "dd_graph_end": [_P, ctypes.POINTER(_P)],
    "dd_graph_launch": [_P, ctypes.c_ulonglong],
    "dd_graph_nodes": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "dd_graph_destroy": [_P],
    "dd_autotune": [_P, _I, _P, _P, _I, ctypes.POINTER(dd_tune_report)],
    "dd_set_tuning": [_P, _I, _I, _I, _I, _I, _I, _I],
    "dd_finalize": [_P],
}

_lib = None


def load():
    """Load libdd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run paper_1112_1243_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name == "dd_last_error" else ctypes.c_int
    _lib = lib
    return lib


def exported_symbols():
    return list(SIGNATURES)
