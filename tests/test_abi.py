"""The C-ABI library builds, loads and exports every entry point that
include/dd.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "dd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dd_[a-z_0-9A-Z]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("dd_init", "dd_apply_D", "dd_apply_D_block", "dd_solve", "dd_det_ratio_estimate",
                     "dd_block_filter", "dd_gauge_update", "dd_workspace_size", "dd_set_workspace",
                     "dd_get_maps", "dd_status", "dd_last_error", "dd_finalize"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1112_1243_gb300 import build, _lib
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    # the Python binding covers the same set, with the same names
    assert sorted(_lib.SIGNATURES) == declared_symbols()
    _lib.load()


def test_binding_constants_match_the_header():
    """Every integer constant that include/dd.h defines has the same value in
    the Python binding (precisions, modes, purposes, error codes)."""
    from paper_1112_1243_gb300 import _lib
    text = open(os.path.join(ROOT, "include", "dd.h")).read()
    defs = re.findall(r"#define\s+(DD_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", text)
    assert len(defs) > 30
    for name, value in defs:
        assert hasattr(_lib, name), name
        assert getattr(_lib, name) == int(value), name


def _noalloc(lib, dims, block, kappa=0.13, bc=-1, cm=3, tol=1e-12, U=None, ln=None):
    import numpy as np
    d = (ctypes.c_int * 4)(*dims)
    b = (ctypes.c_int * 4)(*block)
    buf = np.zeros(4)   # stands in for device pointers: these calls return before any device access
    p = ctypes.c_void_p(buf.ctypes.data)
    return lib.dd_block_ratios_noalloc(d, b, kappa, bc, cm, p if U is None else U, p, 1, 2, tol,
                                       p if ln is None else ln, None)


def test_argument_errors_are_returned_before_any_device_work():
    """dd_init and dd_block_ratios_noalloc validate on the host and return
    their documented error codes without touching a device (runs without a GPU)."""
    from paper_1112_1243_gb300 import build, _lib
    build.build()
    lib = _lib.load()

    def init(dims, block, kappa=0.13, bc=-1):
        p = _lib.dd_params()
        lib.dd_default_params(ctypes.byref(p))
        for a in range(4):
            p.dims[a], p.block[a] = dims[a], block[a]
        p.kappa, p.bc_time = kappa, bc
        h = ctypes.c_void_p()
        return lib.dd_init(ctypes.byref(h), ctypes.byref(p), None)

    assert init((8, 8, 8, 6), (4, 4, 4, 4)) == _lib.DD_ERR_INVALID_ARG       # block does not divide
    assert init((8, 8, 8, 12), (4, 4, 4, 4)) == _lib.DD_ERR_INVALID_ARG      # three blocks along time
    assert init((8, 8, 8, 8), (4, 4, 4, 4), kappa=0.0) == _lib.DD_ERR_INVALID_ARG
    assert init((8, 8, 8, 8), (4, 4, 4, 4), bc=0) == _lib.DD_ERR_INVALID_ARG
    # 12 V >= 2^32: the noise element word would wrap
    assert init((64, 64, 64, 2048), (8, 8, 8, 8)) == _lib.DD_ERR_UNSUPPORTED
    assert _noalloc(lib, (64, 64, 64, 2048), (8, 8, 8, 8)) == _lib.DD_ERR_UNSUPPORTED
    # allocation-free entry point: arguments, and a block too large for its scratch array
    assert _noalloc(lib, (8, 8, 8, 8), (4, 4, 4, 4), kappa=0.0) == _lib.DD_ERR_INVALID_ARG
    assert _noalloc(lib, (8, 8, 8, 8), (4, 4, 4, 4), cm=0) == _lib.DD_ERR_INVALID_ARG
    assert _noalloc(lib, (8, 8, 8, 8), (4, 4, 4, 4), cm=4) == _lib.DD_ERR_INVALID_ARG
    assert _noalloc(lib, (8, 8, 8, 8), (4, 4, 4, 4), bc=0) == _lib.DD_ERR_INVALID_ARG
    assert _noalloc(lib, (8, 8, 8, 8), (4, 4, 4, 4), tol=0.0) == _lib.DD_ERR_INVALID_ARG
    assert _noalloc(lib, (8, 8, 8, 8), (4, 4, 4, 4), ln=ctypes.c_void_p(0)) == _lib.DD_ERR_INVALID_ARG
    assert _noalloc(lib, (8, 8, 8, 12), (4, 4, 4, 4)) == _lib.DD_ERR_INVALID_ARG
    # 16^4 sites x 1248 B per site exceed the 64 MiB scratch array
    assert _noalloc(lib, (32, 32, 32, 32), (16, 16, 16, 16)) == _lib.DD_ERR_UNSUPPORTED
