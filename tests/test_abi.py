"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/lqcd.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_ ]+\**\s*\**(lqcd_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_1612_06424_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "lqcd_factorized_propagator" in names and "lqcd_link_force" in names and len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib

    from paper_1612_06424_gb300 import lqcd

    monkeypatch.setattr(lqcd, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(lqcd, "_lib", None)
    try:
        lqcd.lib()
        raised = False
    except ImportError:
        raised = True
    assert raised
    importlib.reload(lqcd)
