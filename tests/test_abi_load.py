"""The C-ABI library builds, loads and exports every function include/ed.h declares (CPU only)."""
import ctypes
import os
import re

from tests._gpu import ROOT, ensure_built


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ed.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*int\s+(ed_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_core_calls():
    names = declared_functions()
    for n in ("ed_ctx_create", "ed_sector_create", "ed_apply_h", "ed_lanczos", "ed_greens_cf"):
        assert n in names


def test_library_exports_every_declared_symbol():
    ed = ensure_built()
    L = ctypes.CDLL(ed.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    # the binding wraps exactly the declared set
    assert sorted(ed.EXPORTED) == declared_functions()


def test_abi_version_and_error_path_without_gpu():
    ed = ensure_built()
    assert ed.lib().ed_abi_version() == ed.ABI_VERSION == 3
    # NULL output handle is rejected before any device work
    st = ed.lib().ed_ctx_create(0, 0, None)
    assert st == ed.ED_ERR_INVALID
    assert "NULL" in ed.last_error()
