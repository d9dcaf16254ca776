"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/ssa.h (no GPU needed: nothing is called)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(ssa_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    from paper_0911_4498_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built):
    import ctypes
    lib = ctypes.CDLL(built)
    decl = _declared()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_covers_header():
    from paper_0911_4498_gb300 import _lib
    assert set(_declared()) <= set(_lib.exported_symbols())


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_0911_4498_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError):
        _lib.lib()
