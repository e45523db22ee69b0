"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every entry point that include/ldl.h declares (no compute calls)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ldl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ldl_[a-z0-9_]+)\s*\(", text)))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs nvcc")
def test_library_builds_and_exports_every_declared_symbol():
    from paper_2502_18497_gb300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "ldl_create" in names and "ldl_apply_batch" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_2502_18497_gb300 import ldl
    assert sorted(ldl.exported_symbols()) == _declared()


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs nvcc")
@pytest.mark.parametrize("bins", [(40, 96, 1024, 2048), (24, 20, 1024, 2048), (24, 96, 2048, 2048),
                                  (24, 96, 1024, 4096)])
def test_create_rejects_sweep_bins_beyond_the_tables(bins):
    """Degree-bin bounds above a bin's table limit, or decreasing, are rejected
    with LDL_E_INVALID before any device work (so this runs without a GPU)."""
    import numpy as np
    from paper_2502_18497_gb300 import ldl
    lib = ldl.load()
    p = ldl.make_params(directed=True, bin_deg=bins)
    rp = np.array([0, 1, 2], np.int64)
    col = np.array([1, 0], np.int32)
    w = np.array([1, 1], np.int32)
    h = ctypes.c_void_p()
    st = lib.ldl_create(ctypes.byref(p), 2, 2, rp.ctypes.data, col.ctypes.data, w.ctypes.data, ctypes.byref(h))
    assert st == ldl.LDL_E_INVALID and not h.value
    assert b"bins" in lib.ldl_last_error(None)
