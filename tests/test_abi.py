"""CPU checks of the C-ABI library: it builds, loads and exports every symbol
that include/lds.h declares.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "lds.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lds_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_and_exports_header_symbols():
    from paper_2504_10937_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_has_no_fallback(monkeypatch):
    from paper_2504_10937_gb300 import lds
    lib = lds.load()
    assert lds.version().startswith("liblds")
    # a missing library is an error, never a silent fallback
    monkeypatch.setattr(lds, "_lib", None)
    monkeypatch.setattr(lds, "LIB_PATH", os.path.join(ROOT, "does_not_exist.so"))
    with pytest.raises(RuntimeError):
        lds.load()
