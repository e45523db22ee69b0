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
