"""The C-ABI library loads and exports every symbol include/hm.h declares
(no compute call is made without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "hm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hm_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    so = os.path.join(ROOT, "paper_2109_04129_gb300", "libhmps.so")
    if not os.path.exists(so):
        import __graft_entry__
        __graft_entry__.build()
    return ctypes.CDLL(so)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 16
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_all_symbols():
    import paper_2109_04129_gb300 as hp
    assert sorted(hp.SYMBOLS) == _declared()
    assert sorted(hp.exported_symbols()) == _declared()


def test_status_strings_and_defaults(lib):
    import paper_2109_04129_gb300 as hp
    lib.hm_status_string.restype = ctypes.c_char_p
    assert lib.hm_status_string(0) == b"ok"
    assert b"Eq. 45" in lib.hm_status_string(100)
    p = hp.default_params()
    assert p.n_terms == 2 and p.leaf_max == 64 and abs(p.aca_tol - 1e-4) < 1e-18
    assert p.precision == hp.HM_FP64 and p.fill == hp.HM_FILL_FULL


def test_null_arguments_rejected(lib):
    import paper_2109_04129_gb300 as hp
    assert lib.hm_power_series_solve(None, None, None, 1) == hp.HM_ERR_INVALID
    assert lib.hm_destroy(None) == hp.HM_OK
    h = ctypes.c_void_p()
    assert lib.hm_import(None, None, ctypes.byref(h)) == hp.HM_ERR_INVALID
    assert lib.hm_solve_grouped(None, None, None, None, 1) == hp.HM_ERR_INVALID
    arr = (ctypes.c_void_p * 1)(None)
    nr = (ctypes.c_int * 1)(1)
    assert lib.hm_solve_grouped(arr, arr, arr, nr, 1) == hp.HM_ERR_INVALID
    assert lib.hm_solve_grouped(arr, arr, arr, nr, 0) == hp.HM_ERR_INVALID


def test_binding_fails_loudly_without_library(tmp_path):
    """A copy of the binding with no libhmps.so beside it refuses to import:
    there is no CPU fallback."""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "hmps_copy"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_2109_04129_gb300", "__init__.py"), pkg / "__init__.py")
    r = subprocess.run([sys.executable, "-c", "import hmps_copy"], cwd=tmp_path,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "native library not built" in r.stderr
