"""The C-ABI library loads and exports every entry point include/adlbr.h
declares (no GPU needed: nothing is called but adlbr_version)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(adlbr_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_library_exports_declared_symbols():
    from paper_1301_3925_gb300 import build
    build.build()
    import ctypes
    L = ctypes.CDLL(build.LIB)
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_declared_symbols():
    from paper_1301_3925_gb300 import adlbr
    names = _declared()
    missing = [n for n in names if not hasattr(adlbr, n)]
    assert not missing, missing
    assert "sm_103a" in adlbr.adlbr_version()
