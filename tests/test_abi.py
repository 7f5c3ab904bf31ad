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
