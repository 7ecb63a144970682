"""The C-ABI library loads on the CPU host and exports every declared symbol."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(phl_[a-z0-9_]+)\s*\(", txt)))


def test_library_builds_and_exports_every_declared_symbol():
    import __graft_entry__ as ge
    ge.build()
    import ctypes
    import paper_2604_12672_gb300 as P
    lib = ctypes.CDLL(P.LIB_PATH)
    names = _declared("phl.h")
    assert "phl_step" in names and "phl_create_grid" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_2604_12672_gb300 as P
    names = _declared("phl.h")
    assert sorted(P._SIGS) == names


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    import paper_2604_12672_gb300 as P
    monkeypatch.setattr(P, "_lib", None)
    monkeypatch.setattr(P, "LIB_PATH", str(tmp_path / "libphl.so"))
    with pytest.raises(RuntimeError):
        P.lib()


def test_package_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2604_12672_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "oracle.h" not in txt and "liboracle" not in txt, f
